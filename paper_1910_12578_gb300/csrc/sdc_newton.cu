// sdc_newton.cu -- kernels of the implicit reaction update (paper section 2,
// Eq. sdc:general: implicit in R) and of the reactive source R(U).
#include "sdc_launch.h"
#include "sdc_newton.cuh"

namespace sdcd {

constexpr int NEWTON_BLOCK = 128;

template <int NS, int TOPO, typename MT>
__global__ void __launch_bounds__(NEWTON_BLOCK)
newton_kernel(NetParams P, NewtonCfg cfg, long long N, int dim, const double* __restrict__ rhs,
              const double* guess, double* Uout, double* __restrict__ Rout, const double* __restrict__ dt_dev,
              double dt_frac, double dtm_host, int* __restrict__ zone_status, int* __restrict__ zone_iters,
              DevStats* __restrict__ stats) {
    constexpr int NW = NS + 1;
    __shared__ unsigned int hist[64];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = z < N;
    int iters = 0, status = ZONE_OK;
    if (active) {
        const double dtm = dt_dev ? (*dt_dev) * dt_frac : dtm_host;
        const double rho = rhs[z];
        double mom[3] = {0.0, 0.0, 0.0}, m2 = 0.0;
        for (int d = 0; d < dim; d++) {
            mom[d] = rhs[(1 + d) * N + z];
            m2 += mom[d] * mom[d];
        }
        double rw[NW], w[NW], R[NW];
        const double scale = rho / guess[z];
#pragma unroll
        for (int r = 0; r < NW; r++) {
            rw[r] = rhs[(1 + dim + r) * N + z];
            w[r] = guess[(1 + dim + r) * N + z] * scale;
        }
        status = newton_zone<NS, TOPO, MT>(P, cfg, rho, m2, rw, dtm, w, R, iters);
        Uout[z] = rho;
        for (int d = 0; d < dim; d++) Uout[(1 + d) * N + z] = mom[d];
#pragma unroll
        for (int r = 0; r < NW; r++) {
            Uout[(1 + dim + r) * N + z] = w[r];
            Rout[r * N + z] = R[r];
        }
        if (zone_status) zone_status[z] = status;
        if (zone_iters) zone_iters[z] = iters;
        atomicAdd(&hist[iters < 63 ? iters : 63], 1u);
    }
    // warp-aggregated totals
    unsigned long long it = active ? (unsigned long long)iters : 0ull;
    unsigned long long fl = (active && status != ZONE_OK) ? 1ull : 0ull;
    unsigned long long nz = active ? 1ull : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        it += __shfl_down_sync(0xffffffffu, it, o);
        fl += __shfl_down_sync(0xffffffffu, fl, o);
        nz += __shfl_down_sync(0xffffffffu, nz, o);
    }
    if ((threadIdx.x & 31) == 0 && nz) {
        atomicAdd(&stats->iters_total, it);
        atomicAdd(&stats->solves, nz);
        if (fl) atomicAdd(&stats->fails, fl);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 64; i += blockDim.x)
        if (hist[i]) atomicAdd(&stats->hist[i], (unsigned long long)hist[i]);
}

template <int NS, int TOPO>
__global__ void __launch_bounds__(NEWTON_BLOCK)
reaction_source_kernel(NetParams P, long long N, int dim, const double* __restrict__ U, double* __restrict__ R) {
    constexpr int NW = NS + 1;
    constexpr int NR = NS - 1;
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const double rho = U[z];
    double m2 = 0.0;
    for (int d = 0; d < dim; d++) {
        const double m = U[(1 + d) * N + z];
        m2 += m * m;
    }
    const double inv_rho = 1.0 / rho;
    const double T = P.gm1 * (U[(1 + dim) * N + z] - 0.5 * m2 * inv_rho) * inv_rho;
    double k[NR], dk[NR], Y[NS], Rz[NW];
    rate_consts<NR>(P, rho, T, k, dk);
#pragma unroll
    for (int i = 0; i < NS; i++) Y[i] = U[(2 + dim + i) * N + z] * (inv_rho * P.inv_mass[i]);
    sources<NS, TOPO>(P, rho, k, Y, Rz);
#pragma unroll
    for (int r = 0; r < NW; r++) R[r * N + z] = Rz[r];
}

// ---------------------------------------------------------------- dispatch
#define SDC_NEWTON_CASES(X) \
    X(2, TOPO_GENERIC)      \
    X(3, TOPO_GENERIC)      \
    X(4, TOPO_GENERIC)      \
    X(5, TOPO_GENERIC)      \
    X(5, TOPO_CHAIN)        \
    X(7, TOPO_CHAIN)        \
    X(13, TOPO_CHAIN)

bool newton_supported(int nspec, int topo) {
#define X(ns, tp) \
    if (nspec == ns && topo == tp) return true;
    SDC_NEWTON_CASES(X)
#undef X
    return false;
}

cudaError_t launch_newton(const NetParams& P, const NewtonCfg& cfg, int prec, long long N, int dim,
                          const double* rhs, const double* guess, double* Uout, double* Rout,
                          const double* dt_dev, double dt_frac, double dtm_host, int* zone_status,
                          int* zone_iters, DevStats* stats, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((N + NEWTON_BLOCK - 1) / NEWTON_BLOCK);
#define X(ns, tp)                                                                                         \
    if (P.nspec == ns && P.topo == tp) {                                                                  \
        if (prec == 0)                                                                                    \
            newton_kernel<ns, tp, double><<<grid, NEWTON_BLOCK, 0, st>>>(P, cfg, N, dim, rhs, guess, Uout,  \
                                                                         Rout, dt_dev, dt_frac, dtm_host, \
                                                                         zone_status, zone_iters, stats); \
        else                                                                                              \
            newton_kernel<ns, tp, float><<<grid, NEWTON_BLOCK, 0, st>>>(P, cfg, N, dim, rhs, guess, Uout,   \
                                                                        Rout, dt_dev, dt_frac, dtm_host,  \
                                                                        zone_status, zone_iters, stats);  \
        return cudaGetLastError();                                                                        \
    }
    SDC_NEWTON_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_reaction_source(const NetParams& P, long long N, int dim, const double* U, double* R,
                                   cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((N + NEWTON_BLOCK - 1) / NEWTON_BLOCK);
#define X(ns, tp)                                                                              \
    if (P.nspec == ns && P.topo == tp) {                                                       \
        reaction_source_kernel<ns, tp><<<grid, NEWTON_BLOCK, 0, st>>>(P, N, dim, U, R);        \
        return cudaGetLastError();                                                             \
    }
    SDC_NEWTON_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace sdcd
