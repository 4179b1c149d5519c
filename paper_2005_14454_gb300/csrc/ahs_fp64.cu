// ahs_fp64.cu -- the random-phase initial condition of the FP64 precision mode
// (Sec. 2; SplitMix64 counter-based phases as in the float32 init, stored in
// double).  The FP64 step is the tiled kernel of ahs_step.cu instantiated in
// double (launch_step64).
#include "ahs_device.cuh"

namespace eng {
namespace {

__global__ void init_fp64(double *pr, double *pim, size_t V, uint64_t seed, double sigma)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < V; i += (size_t)gridDim.x * blockDim.x) {
        uint64_t z = (seed ^ splitmix64_device((uint64_t)i));
        const double u = (double)(splitmix64_device(z) >> 11) * (1.0 / 9007199254740992.0);
        double s, c;
        sincos(__dmul_rn(2.0 * kPiD, u), &s, &c);
        pr[i] = __dmul_rn(sigma, c);
        pim[i] = __dmul_rn(sigma, s);
    }
}

}  // namespace

cudaError_t launch_init_fp64(double *pr, double *pim, int N, uint64_t seed, double sigma, cudaStream_t st)
{
    const size_t V = (size_t)N * N * N;
    const size_t want = (V + 255) / 256;
    init_fp64<<<(int)(want < (size_t)152 * 64 ? want : (size_t)152 * 64), 256, 0, st>>>(pr, pim, V, seed, sigma);
    return cudaGetLastError();
}

}  // namespace eng
