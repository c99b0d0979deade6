// sdc_newton.cu -- kernels of the implicit reaction update (paper section 2,
// Eq. sdc:general: implicit in R) and of the reactive source R(U).
#include "sdc_launch.h"
#include "sdc_newton.cuh"
#include "sdc_newton_group.cuh"

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

// L lanes per zone (alpha chain); zone state in dynamic shared memory
constexpr int GROUP_L = 4;

template <int NS, typename MT, int L>
__global__ void __launch_bounds__(NEWTON_BLOCK)
newton_group_kernel(NetParams P, NewtonCfg cfg, long long N, int dim, const double* __restrict__ rhs,
                    const double* guess, double* Uout, double* __restrict__ Rout, const double* __restrict__ dt_dev,
                    double dt_frac, double dtm_host, int* __restrict__ zone_status, int* __restrict__ zone_iters,
                    DevStats* __restrict__ stats) {
    using Lay = GroupLayout<NS, MT>;
    constexpr int NW = NS + 1;
    constexpr int RL = (NW + L - 1) / L;
    extern __shared__ double gsm[];
    __shared__ unsigned int hist[64];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x % L;
    const int gz = threadIdx.x / L;  // zone of this group within the block
    const unsigned mask = ((1u << L) - 1u) << ((threadIdx.x & 31) & ~(L - 1));
    const long long z = (long long)blockIdx.x * (NEWTON_BLOCK / L) + gz;
    const bool active = z < N;
    double* zs = gsm + (size_t)gz * Lay::STRIDE;
    int iters = 0, status = ZONE_OK;
    if (active) {
        const double dtm = dt_dev ? (*dt_dev) * dt_frac : dtm_host;
        const double rho = rhs[z];
        double mom[3] = {0.0, 0.0, 0.0}, m2 = 0.0;
        for (int d = 0; d < dim; d++) {
            mom[d] = rhs[(1 + d) * N + z];
            m2 += mom[d] * mom[d];
        }
        const double scale = rho / guess[z];
        double rw_rows[RL];
#pragma unroll
        for (int t = 0; t < RL; t++) {
            const int row = lane + L * t;
            rw_rows[t] = 0.0;
            if (row < NW) {
                rw_rows[t] = rhs[(1 + dim + row) * N + z];
                zs[Lay::O_W + row] = guess[(1 + dim + row) * N + z] * scale;
            }
        }
        __syncwarp(mask);
        status = newton_zone_group<NS, MT, L>(P, cfg, mask, lane, zs, rho, m2, rw_rows, dtm, iters);
        if (lane == 0) {
            Uout[z] = rho;
            for (int d = 0; d < dim; d++) Uout[(1 + d) * N + z] = mom[d];
            if (zone_status) zone_status[z] = status;
            if (zone_iters) zone_iters[z] = iters;
            atomicAdd(&hist[iters < 63 ? iters : 63], 1u);
        }
#pragma unroll
        for (int t = 0; t < RL; t++) {
            const int row = lane + L * t;
            if (row < NW) {
                Uout[(1 + dim + row) * N + z] = zs[Lay::O_W + row];
                Rout[row * N + z] = zs[Lay::O_G + row];
            }
        }
    }
    const bool lead = active && lane == 0;
    unsigned long long it = lead ? (unsigned long long)iters : 0ull;
    unsigned long long fl = (lead && status != ZONE_OK) ? 1ull : 0ull;
    unsigned long long nz = lead ? 1ull : 0ull;
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

template <int NS, typename MT>
constexpr size_t group_smem() {
    return sizeof(double) * (size_t)GroupLayout<NS, MT>::STRIDE * (NEWTON_BLOCK / GROUP_L);
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
    X(7, TOPO_CHAIN)

// the 13-species chain: a group of lanes per zone (newton_group_kernel)
bool newton_group_case(int nspec, int topo) { return nspec == 13 && topo == TOPO_CHAIN; }

cudaError_t newton_prepare(int nspec, int topo) {
    if (!newton_group_case(nspec, topo)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(newton_group_kernel<13, double, GROUP_L>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)group_smem<13, double>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(newton_group_kernel<13, float, GROUP_L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)group_smem<13, float>());
}

bool newton_supported(int nspec, int topo) {
    if (newton_group_case(nspec, topo)) return true;
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
    if (P.nspec == 13 && P.topo == TOPO_CHAIN) {
        constexpr int ZPB = NEWTON_BLOCK / GROUP_L;
        const unsigned ggrid = (unsigned)((N + ZPB - 1) / ZPB);
        if (prec == 0)
            newton_group_kernel<13, double, GROUP_L><<<ggrid, NEWTON_BLOCK, group_smem<13, double>(), st>>>(
                P, cfg, N, dim, rhs, guess, Uout, Rout, dt_dev, dt_frac, dtm_host, zone_status, zone_iters, stats);
        else
            newton_group_kernel<13, float, GROUP_L><<<ggrid, NEWTON_BLOCK, group_smem<13, float>(), st>>>(
                P, cfg, N, dim, rhs, guess, Uout, Rout, dt_dev, dt_frac, dtm_host, zone_status, zone_iters, stats);
        return cudaGetLastError();
    }
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
    if (newton_group_case(P.nspec, P.topo)) {
        reaction_source_kernel<13, TOPO_CHAIN><<<grid, NEWTON_BLOCK, 0, st>>>(P, N, dim, U, R);
        return cudaGetLastError();
    }
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
