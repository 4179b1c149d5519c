// ahs_internal.cuh -- shared declarations of the GB300 engine (kernels + host ABI).
//
// Lattice Abelian-Higgs evolution of Correia & Martins (arXiv:2005.14454), Sec. 2:
// staggered leapfrog (Eqs. 7-10), covariant Laplacian (Eq. 14), plaquettes
// (Eqs. 15-16), diagnostics (Eqs. diagxi, diagvel).  Storage is float32 SoA,
// site index x + N*(y + N*z).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "ahs.h"

namespace eng {

// ---- reduction slots of one measurement (per-block FP64 partials) ----------
enum {
    Q_K = 0, Q_G, Q_V, Q_EL, Q_B, Q_L, Q_KL, Q_GL, Q_PL, Q_RL,  // site sums
    Q_G2,      // sum of squared Gauss residual
    Q_GMAX,    // max |Gauss residual|
    Q_WIND,    // sum |W_ij| over plaquettes
    Q_NF,      // sites with a non-finite diagnostic
    NQ = 16
};
constexpr int NSUM = 11;   // slots Q_K..Q_G2 are plain sums

// Device pointers of one step.  Every field is double buffered: the step reads
// phi^n, theta^n, Pi^{n-1/2}, E^{n-1/2} from one buffer and writes phi^{n+1},
// theta^{n+1}, Pi^{n+1/2}, E^{n+1/2} into the other, so no thread ever reads a
// value another thread of the same launch has already replaced.
struct StepPtrs {
    const float *pr, *pim, *tx, *ty, *tz, *qr, *qi, *ex, *ey, *ez;
    float *pr1, *pim1, *tx1, *ty1, *tz1, *qr1, *qi1, *ex1, *ey1, *ez1;
    // compensated precision only: low words of Pi and E (value = high + low)
    const float *qrl, *qil, *exl, *eyl, *ezl;
    float *qrl1, *qil1, *exl1, *eyl1, *ezl1;
};

// FP64 precision mode: the same fields in double
struct StepPtrs64 {
    const double *pr, *pim, *tx, *ty, *tz, *qr, *qi, *ex, *ey, *ez;
    double *pr1, *pim1, *tx1, *ty1, *tz1, *qr1, *qi1, *ex1, *ey1, *ez1;
};

// Per-step coefficients, computed in FP64 on the host from the step index and
// rounded once to float32.
//   Pi^{n+1/2} = cpi Pi + kpi_lap (sum_i [U phi(x+i) + U^* phi(x-i)] - 6 phi)
//                - kpi_pot (|phi|^2 - sigma^2) phi                       (Eq. 7)
//   E_i^{n+1/2} = ce E_i + ke_curl (curl of sin alpha)_i + ke_cur J_i     (Eq. 8)
//   phi += dphi Pi, theta_i += dtheta E_i                               (Eqs. 9-10)
struct StepCoef {
    float cpi, kpi_lap, kpi_pot, sigma2;
    float ce, ke_curl, ke_cur;
    float dphi, dtheta;
    int wrap;
    // measurement factors (Eqs. diagxi, diagvel and the Gauss residual)
    float m_grad;   // 1/dx^2
    float m_pot;    // lambda0 c / 4
    float m_el;     // 1/(8 e0^2 c): 1/(2 e0^2 c) times the 1/4 of squaring a mean of two
    float m_mag;    // 1/(e0^2 c dx^4)
    float m_gauss;  // 2 e0^2 kappa_{n-1}
    float inv_dx;
    int gauss;      // 1: a measuring step computes the Gauss residual itself; 0: an
                    // earlier launch (launch_gauss) wrote it into the partial rows
};

// the coefficients of StepCoef without rounding, for the FP64 mode
struct StepCoef64 {
    double cpi, kpi_lap, kpi_pot, sigma2;
    double ce, ke_curl, ke_cur;
    double dphi, dtheta;
    int wrap;
    double m_grad, m_pot, m_el, m_mag, m_gauss, inv_dx;
    int gauss;
};

// Scalars the final reduction needs to turn sums into an observable record.
struct ObsScalars {
    int64_t step;
    double tau, a, dx, sites, volume, mu;
};

// Launchers (ahs_kernels.cu).  All take the stream they run on.
cudaError_t launch_init(float *pr, float *pim, int N, uint64_t seed, double sigma, cudaStream_t st);
// Launch shape of the z-marching step kernel: tile height (4, 8 or 16 rows of 32
// sites), z-chunk per CTA, and the number of CTAs (= rows of measurement partials).
struct StepShape {
    int by, dz, blocks;
};
StepShape step_shape(int N, int tile_y, int zchunk);   // tile_y/zchunk 0: automatic
// the shape of a measuring launch (and of the Gauss pass that goes with it): tile
// height 4, 8 or 16 (0: automatic, 4)
StepShape measure_shape(int N, int tile_y, int zchunk);
cudaError_t launch_step(const StepPtrs &p, const StepCoef &k, int N, const StepShape &sh, bool measure, bool store,
                        double *partials, cudaStream_t st, bool compensated = false);
// FP64 precision: the tiled step in double, 8-row tiles (sh.by must be 8)
// The Gauss residual alone (the Q_G2 and Q_GMAX slots of the partial rows of the
// measuring launch of the same shape, in the same order of operations), for
// measuring steps whose launch overwrites E in place.
cudaError_t launch_gauss(const StepPtrs &p, const StepCoef &k, int N, const StepShape &sh, double *partials,
                         cudaStream_t st);
// Two plain float32 steps n -> n+2 in one pass (temporal blocking): k1, k2 are
// the coefficients of steps n and n+1; reads the time-n buffer, writes the other.
// 32 x 8 tiles, Dz planes per CTA.
cudaError_t launch_step_two(const StepPtrs &p, const StepCoef &k1, const StepCoef &k2, int N, int Dz,
                            cudaStream_t st);
cudaError_t launch_step64(const StepPtrs64 &p, const StepCoef64 &k, int N, const StepShape &sh, bool measure,
                          bool store, double *partials, cudaStream_t st);
cudaError_t launch_init_fp64(double *pr, double *pim, int N, uint64_t seed, double sigma, cudaStream_t st);
cudaError_t launch_reduce(const double *partials, int nblocks, const ObsScalars &sc,
                          ahs_obs_t *rec, cudaStream_t st);
cudaError_t launch_windings(const float *pr, const float *pim, const float *tx, const float *ty,
                            const float *tz, int N, int8_t *W, cudaStream_t st);
cudaError_t launch_gather_box(const float *const *planes, int nplanes, int N, int x0, int y0, int z0,
                              int nx, int ny, int nz, float *dst, cudaStream_t st);

// ---- batched ensembles: many lattices advanced by one persistent launch -------
// One tile of work (the 32 x BY column at (x0, y0), planes [z0, zend)) of member
// `member`; its measurement partials go to the row with the tile's index.
struct BatchTile {
    int member, x0, y0, z0, zend, pad;
};
// A member lattice: its two field buffers (base: buffer 0 Re phi; the twenty
// planes of N^3 floats follow each other, buffer 1 starting at plane 10), side,
// last step, and its rows of measurement partials.  Members have 20 N^3 < 2^32.
struct BatchMember {
    const float *base;
    int N, row0, nrows, pad;
    int64_t n_end;
};
// Everything one batched step launch reads.  The step index is *counter + dn
// (dn is fixed when a launch is recorded into a graph); coefficients come from a
// table computed on the host in FP64, coef[member * coef_stride + n].
struct BatchLaunch {
    const BatchTile *tiles;
    int ntiles;
    const int *live;          // live[n]: tiles of members still running at step n (a prefix of the list)
    int *tickets;             // tickets[n]: next unclaimed tile of step n (zero before the step)
    const BatchMember *members;
    int nmembers;
    const StepCoef *coef;
    int coef_stride;
    const int64_t *counter;
    double *partials;
};
cudaError_t launch_batch_step(const BatchLaunch &L, int by, int dn, bool measure, int grid, cudaStream_t st);
int batch_grid(int by, bool measure);   // resident CTAs of the persistent launch
// the plain step of members of even side on paired 64 x 8 tiles (tiles of the list
// start at x0 multiples of 64), and its resident CTAs
cudaError_t launch_batch_pair_step(const BatchLaunch &L, int dn, int grid, cudaStream_t st);
int batch_pair_grid();
// per-member measurement record of step *counter + dn when that step is a
// measurement step of the member: records[m * rcap + n / every]
cudaError_t launch_batch_reduce(const double *partials, const BatchMember *members, int nmembers,
                                const ObsScalars *obs, int obs_stride, const int64_t *counter, int dn, int every,
                                ahs_obs_t *records, int rcap, cudaStream_t st);
cudaError_t launch_advance(int64_t *counter, int64_t delta, cudaStream_t st);

// counters of the bounds-check build (ahs_bounds_check): the out-of-range indices
// the kernels of ahs_step.cu and of ahs_step2.cu counted on the current device;
// op 0 reads, 1 reads and zeroes, 2 first runs the self-test launch.
// cudaErrorNotSupported in the production build.
cudaError_t bounds_errors_step(unsigned long long *count, int op);
cudaError_t bounds_errors_step2(unsigned long long *count, int op);

// error state of the C ABI (ahs_last_error / ahs_last_error_message)
int report_error(int code, const char *msg);
int report_ok();

}  // namespace eng
