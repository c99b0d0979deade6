// sdc_newton.cu -- kernels of the implicit reaction update (paper section 2,
// Eq. sdc:general: implicit in R) and of the reactive source R(U).
#include "sdc_launch.h"
#include "sdc_newton.cuh"
#include "sdc_newton_group.cuh"

namespace sdcd {

constexpr int NEWTON_BLOCK = 128;

// Resident blocks per SM the one-zone-per-thread kernels ask the register
// allocator for: three (168 registers a thread, twelve warps per SM) in every
// precision.  The float-pair solve's FP32 work is a chain of dependent
// operations, and the FP64 and FP32-Jacobian solves keep their FP64 pipe busier
// with the extra warps, though their 13-species kernels then spill more.
// Measured at 256^3, 13 species, Newton per step: float pairs 219.7 (two blocks)
// -> 178.2 ms; FP64 217.6 (two) -> 210.3 (three) -> 213.0 ms (four); FP32
// Jacobian 155.3 (two) -> 141.3 ms; 7 species unchanged.
template <typename MT>
constexpr int newton_min_blocks() {
    return 3;
}

// Load zone z into a solver state and evaluate it.  The start: with Rpred
// (R^{m+1,(k)} of the sweep), the explicit predictor rhs + dt_m R^{m+1,(k)}
// where it has a positive temperature and no mass fraction below -0.01,
// otherwise (and without Rpred) the guess carried to the density of the rhs.
// The predictor is formed with separate roundings (no fused multiply-add), as
// the oracle forms it.
template <int NS, int TOPO>
__device__ __forceinline__ void load_zone(ZoneState<NS>& S, const NetParams& P, long long N, int dim, long long z,
                                          const double* __restrict__ rhs, const double* guess,
                                          const double* __restrict__ Rpred, double dtm, double* mom,
                                          const double* anchor) {
    constexpr int NW = NS + 1;
    const double rho = rhs[z];
    double m2 = 0.0;
    for (int d = 0; d < 3; d++) mom[d] = 0.0;
    for (int d = 0; d < dim; d++) {
        mom[d] = rhs[(1 + d) * N + z];
        m2 += mom[d] * mom[d];
    }
    double rw[NW];
#pragma unroll
    for (int r = 0; r < NW; r++) rw[r] = rhs[(1 + dim + r) * N + z];
    S.rwp = rhs + (1 + dim) * N + z;
    S.rws = N;
    // 1/rho, the kinetic energy and the floor -0.01 rho, formed once for the start
    // test and the solve
    const double ir = rcp_nr(rho);
    const double ke = 0.5 * m2 * ir;
    const double mr = -XMARGIN * rho;
    bool pred = false;
    double Tw = 0.0;
    if (Rpred) {
#pragma unroll
        for (int r = 0; r < NW; r++) S.w[r] = __dadd_rn(rw[r], __dmul_rn(dtm, Rpred[r * N + z]));
        Tw = P.gm1 * (S.w[0] - ke) * ir;
        pred = positive_finite(Tw);
        // rho X_i >= -0.01 rho, compared on the integer pipe
        const long long floor_x = ordered_bits(mr);
#pragma unroll
        for (int i = 0; i < NS; i++) pred = pred && (ordered_bits(S.w[1 + i]) >= floor_x);
    }
    if (!pred) {
        Tw = 0.0;
        const double scale = rho / guess[z];
#pragma unroll
        for (int r = 0; r < NW; r++) S.w[r] = guess[(1 + dim + r) * N + z] * scale;
    }
    zone_init<NS, TOPO>(S, P, rw, rho, ir, ke, mr, Tw, dtm, anchor, N, z);
}

// Store the solution and R of a finished zone.
template <int NS, int TOPO>
__device__ __forceinline__ void store_zone(const ZoneState<NS>& S, const NetParams& P, long long N, int dim,
                                           long long z, const double* mom, double* Uout, double* __restrict__ Rout,
                                           int* __restrict__ zone_status, int* __restrict__ zone_iters) {
    constexpr int NW = NS + 1;
    double R[NW];
    zone_source<NS, TOPO>(S, P, R);
    Uout[z] = S.rho;
    for (int d = 0; d < dim; d++) Uout[(1 + d) * N + z] = mom[d];
#pragma unroll
    for (int r = 0; r < NW; r++) {
        Uout[(1 + dim + r) * N + z] = S.w[r];
        Rout[r * N + z] = R[r];
    }
    if (zone_status) zone_status[z] = S.status;
    if (zone_iters) zone_iters[z] = S.iters;
}

// One zone per thread, a static grid over the zones.
template <int NS, int TOPO, typename MT>
__global__ void __launch_bounds__(NEWTON_BLOCK, newton_min_blocks<MT>())
newton_kernel(const __grid_constant__ NetParams P, NewtonCfg cfg, long long N, int dim, const double* __restrict__ rhs,
              const double* guess, const double* __restrict__ Rpred, double* Uout, double* __restrict__ Rout,
              const double* __restrict__ dt_dev,
              double dt_frac, double dtm_host, int* __restrict__ zone_status, int* __restrict__ zone_iters,
              DevStats* __restrict__ stats) {
    __shared__ unsigned int hist[64];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = z < N;
    int iters = 0, status = ZONE_OK;
    if (active) {
        const double dtm = dt_dev ? (*dt_dev) * dt_frac : dtm_host;
        ZoneState<NS> S;
        S.lop = newton_floor_smem<NS, MT>();
        S.los = (int)blockDim.x;
        double mom[3];
        load_zone<NS, TOPO>(S, P, N, dim, z, rhs, guess, Rpred, dtm, mom, cfg.anchor);
        while (!S.done) zone_iterate<NS, TOPO, MT>(S, P, cfg, dtm);
        store_zone<NS, TOPO>(S, P, N, dim, z, mom, Uout, Rout, zone_status, zone_iters);
        iters = S.iters;
        status = S.status;
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

// Persistent grid fed by a device work queue: every lane owns one zone's
// solve; when it finishes, the lane stores it and takes the next zone from the
// queue (one atomic per warp refill), so zones that need many iterations do
// not hold the other lanes of their warp idle.  Each zone's arithmetic is the
// same as in newton_kernel, so results agree bit for bit.
template <int NS, int TOPO, typename MT>
__global__ void __launch_bounds__(NEWTON_BLOCK, newton_min_blocks<MT>())
newton_queue_kernel(const __grid_constant__ NetParams P, NewtonCfg cfg, long long N, int dim, const double* __restrict__ rhs,
                    const double* guess, const double* __restrict__ Rpred, double* Uout, double* __restrict__ Rout,
                    const double* __restrict__ dt_dev,
                    double dt_frac, double dtm_host, int* __restrict__ zone_status, int* __restrict__ zone_iters,
                    DevStats* __restrict__ stats, unsigned long long* __restrict__ queue) {
    __shared__ unsigned int hist[64];
    __shared__ unsigned long long blk_iters, blk_solves, blk_fails;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) hist[i] = 0;
    if (threadIdx.x == 0) { blk_iters = 0; blk_solves = 0; blk_fails = 0; }
    __syncthreads();
    const double dtm = dt_dev ? (*dt_dev) * dt_frac : dtm_host;
    const int lane = threadIdx.x & 31;
    ZoneState<NS> S;
    S.lop = newton_floor_smem<NS, MT>();
    S.los = (int)blockDim.x;
    double mom[3];
    long long z = -1;
    bool exhausted = false;
    S.done = true;
    unsigned long long my_iters = 0, my_solves = 0, my_fails = 0;
    for (;;) {
        // lanes without a zone take the next ones from the queue
        const bool need = (z < 0) && !exhausted;
        const unsigned want = __ballot_sync(0xffffffffu, need);
        if (want) {
            unsigned long long base = 0;
            const int leader = __ffs(want) - 1;
            if (lane == leader) base = atomicAdd(queue, (unsigned long long)__popc(want));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (need) {
                const long long zi = (long long)(base + __popc(want & ((1u << lane) - 1u)));
                if (zi < N) {
                    z = zi;
                    load_zone<NS, TOPO>(S, P, N, dim, z, rhs, guess, Rpred, dtm, mom, cfg.anchor);
                } else {
                    exhausted = true;
                }
            }
        }
        if (!__any_sync(0xffffffffu, z >= 0)) break;
        if (z >= 0 && !S.done) zone_iterate<NS, TOPO, MT>(S, P, cfg, dtm);
        if (z >= 0 && S.done) {
            store_zone<NS, TOPO>(S, P, N, dim, z, mom, Uout, Rout, zone_status, zone_iters);
            atomicAdd(&hist[S.iters < 63 ? S.iters : 63], 1u);
            my_iters += (unsigned long long)S.iters;
            my_solves += 1;
            if (S.status != ZONE_OK) my_fails += 1;
            z = -1;
        }
    }
    atomicAdd(&blk_iters, my_iters);
    atomicAdd(&blk_solves, my_solves);
    if (my_fails) atomicAdd(&blk_fails, my_fails);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (blk_solves) {
            atomicAdd(&stats->iters_total, blk_iters);
            atomicAdd(&stats->solves, blk_solves);
        }
        if (blk_fails) atomicAdd(&stats->fails, blk_fails);
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x)
        if (hist[i]) atomicAdd(&stats->hist[i], (unsigned long long)hist[i]);
}

// Persistent grid fed by a device work queue at warp granularity: each warp
// takes the next 32 zones with one atomic, solves them in lockstep as
// newton_kernel does, and takes the next chunk when all 32 are done.  The
// zones of a chunk are neighbours, so their iteration counts are alike (no
// lanes left in other phases of their solves, as in newton_queue_kernel), and
// warps that draw slow chunks do not hold up the rest of the grid.  Each
// zone's arithmetic is that of newton_kernel: results agree bit for bit.
template <int NS, int TOPO, typename MT>
__global__ void __launch_bounds__(NEWTON_BLOCK, newton_min_blocks<MT>())
newton_warpqueue_kernel(const __grid_constant__ NetParams P, NewtonCfg cfg, long long N, int dim, const double* __restrict__ rhs,
                        const double* guess, const double* __restrict__ Rpred, double* Uout,
                        double* __restrict__ Rout,
                        const double* __restrict__ dt_dev, double dt_frac, double dtm_host,
                        int* __restrict__ zone_status, int* __restrict__ zone_iters, DevStats* __restrict__ stats,
                        unsigned long long* __restrict__ queue) {
    __shared__ unsigned int hist[64];
    __shared__ unsigned long long blk_iters, blk_solves, blk_fails;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) hist[i] = 0;
    if (threadIdx.x == 0) { blk_iters = 0; blk_solves = 0; blk_fails = 0; }
    __syncthreads();
    const double dtm = dt_dev ? (*dt_dev) * dt_frac : dtm_host;
    const int lane = threadIdx.x & 31;
    unsigned long long my_iters = 0, my_solves = 0, my_fails = 0;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(queue, 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= (unsigned long long)N) break;  // the same for every lane of the warp
        const long long z = (long long)base + lane;
        if (z < N) {
            ZoneState<NS> S;
            S.lop = newton_floor_smem<NS, MT>();
            S.los = (int)blockDim.x;
            double mom[3];
            load_zone<NS, TOPO>(S, P, N, dim, z, rhs, guess, Rpred, dtm, mom, cfg.anchor);
            while (!S.done) zone_iterate<NS, TOPO, MT>(S, P, cfg, dtm);
            store_zone<NS, TOPO>(S, P, N, dim, z, mom, Uout, Rout, zone_status, zone_iters);
            atomicAdd(&hist[S.iters < 63 ? S.iters : 63], 1u);
            my_iters += (unsigned long long)S.iters;
            my_solves += 1;
            if (S.status != ZONE_OK) my_fails += 1;
        }
    }
    atomicAdd(&blk_iters, my_iters);
    atomicAdd(&blk_solves, my_solves);
    if (my_fails) atomicAdd(&blk_fails, my_fails);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (blk_solves) {
            atomicAdd(&stats->iters_total, blk_iters);
            atomicAdd(&stats->solves, blk_solves);
        }
        if (blk_fails) atomicAdd(&stats->fails, blk_fails);
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x)
        if (hist[i]) atomicAdd(&stats->hist[i], (unsigned long long)hist[i]);
}

// L lanes per zone (alpha chain), GROUP_ZONES zones per block of 32 L threads;
// zone state in dynamic shared memory.  Variant 0: L = 4, variant 1: L = 2
// (half the lanes share each zone's split work, so instructions that every
// lane of a group repeats -- pivot reciprocals, transcendentals, the lane-0
// steps of the back substitution -- occupy half the warp slots per zone).
constexpr int GROUP_ZONES = 32;

template <int NS, typename MT, int L>
__global__ void __launch_bounds__(NEWTON_BLOCK)
newton_group_kernel(NetParams P, NewtonCfg cfg, long long N, int dim, const double* __restrict__ rhs,
                    const double* guess, const double* __restrict__ Rpred, double* Uout, double* __restrict__ Rout,
                    const double* __restrict__ dt_dev,
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
    const long long z = (long long)blockIdx.x * GROUP_ZONES + gz;
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
        double rw_rows[RL];
#pragma unroll
        for (int t = 0; t < RL; t++) {
            const int row = lane + L * t;
            rw_rows[t] = row < NW ? rhs[(1 + dim + row) * N + z] : 0.0;
        }
        // the start: the explicit predictor where admissible (as load_zone), else the guess
        bool pred = false;
        if (Rpred) {
            const double floor_x = -XMARGIN * rho;
            bool ok = true;
#pragma unroll
            for (int t = 0; t < RL; t++) {
                const int row = lane + L * t;
                if (row < NW) {
                    const double v = __dadd_rn(rw_rows[t], __dmul_rn(dtm, Rpred[row * N + z]));
                    zs[Lay::O_W + row] = v;
                    if (row >= 1) ok = ok && !(v < floor_x);
                }
            }
            __syncwarp(mask);
            const double ir = rcp_nr(rho);
            ok = ok && positive_finite(P.gm1 * (zs[Lay::O_W] - 0.5 * m2 * ir) * ir);
            pred = group_all<L>(mask, ok);
        }
        if (!pred) {
            const double scale = rho / guess[z];
#pragma unroll
            for (int t = 0; t < RL; t++) {
                const int row = lane + L * t;
                if (row < NW) zs[Lay::O_W + row] = guess[(1 + dim + row) * N + z] * scale;
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
    return sizeof(double) * (size_t)GroupLayout<NS, MT>::STRIDE * GROUP_ZONES;
}

template <int NS, int TOPO>
__global__ void __launch_bounds__(NEWTON_BLOCK)
reaction_source_kernel(NetParams P, long long N, int dim, const double* __restrict__ U, double* __restrict__ R,
                       double* __restrict__ anchor) {
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
    const double inv_rho = rcp_nr(rho);
    const double T = P.gm1 * (U[(1 + dim) * N + z] - 0.5 * m2 * inv_rho) * inv_rho;
    double k[NR], Y[NS], Rz[NW];
    if constexpr (TOPO == TOPO_CHAIN) {
        // the chain's sources as products of the unknowns: kappa_j = amp_j f_j(T)
        double dfac;
        rate_consts_k<NR>(P, P.amp, T, k, dfac);
#pragma unroll
        for (int i = 0; i < NS; i++) Y[i] = U[(2 + dim + i) * N + z];
        sources_w<NS>(P, k, Y, Rz);
        if (anchor) {
            // the step's rate anchors (NewtonCfg): kappa_j, T and 1/T, or a nan T_a
            // where T is not positive and finite
            const bool ok = positive_finite(T);
#pragma unroll
            for (int j = 0; j < NR; j++) anchor[(long long)j * N + z] = k[j];
            anchor[(long long)NR * N + z] = ok ? T : __longlong_as_double(0x7ff8000000000000ll);
            anchor[(long long)(NR + 1) * N + z] = ok ? dfac : 0.0;
        }
    } else {
        double dk[NR];
        rate_consts<NR>(P, rho, T, k, dk);
#pragma unroll
        for (int i = 0; i < NS; i++) Y[i] = U[(2 + dim + i) * N + z] * (inv_rho * P.inv_mass[i]);
        sources<NS, TOPO>(P, rho, k, Y, Rz);
    }
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

// the 13-species chain: a group of lanes per zone (newton_group_kernel)
bool newton_group_case(int nspec, int topo) { return nspec == 13 && topo == TOPO_CHAIN; }
// the 5- and 7-species chains also have the group kernel, as Newton variant 3
bool newton_small_group_case(int nspec, int topo) { return topo == TOPO_CHAIN && (nspec == 5 || nspec == 7); }

// the float-pair kernels' dynamic shared memory (above the default 48 KB for 13 species)
template <int NS>
cudaError_t pair_prepare() {
    const int b = (int)newton_smem_bytes<NS, f2>(NEWTON_BLOCK);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(newton_kernel<NS, TOPO_CHAIN, f2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  b)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(newton_queue_kernel<NS, TOPO_CHAIN, f2>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, b)) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(newton_warpqueue_kernel<NS, TOPO_CHAIN, f2>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}

cudaError_t newton_prepare(int nspec, int topo) {
    cudaError_t e;
    if (topo == TOPO_CHAIN) {
        e = nspec == 5 ? pair_prepare<5>() : nspec == 7 ? pair_prepare<7>() : nspec == 13 ? pair_prepare<13>()
                                                                                           : cudaSuccess;
        if (e != cudaSuccess) return e;
    }
    if (newton_small_group_case(nspec, topo)) {
        if (nspec == 5) {
            if ((e = cudaFuncSetAttribute(newton_group_kernel<5, double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)group_smem<5, double>())) != cudaSuccess)
                return e;
            return cudaFuncSetAttribute(newton_group_kernel<5, float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)group_smem<5, float>());
        }
        if ((e = cudaFuncSetAttribute(newton_group_kernel<7, double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)group_smem<7, double>())) != cudaSuccess)
            return e;
        return cudaFuncSetAttribute(newton_group_kernel<7, float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)group_smem<7, float>());
    }
    if (!newton_group_case(nspec, topo)) return cudaSuccess;
    const int sd = (int)group_smem<13, double>(), sf = (int)group_smem<13, float>();
    if ((e = cudaFuncSetAttribute(newton_group_kernel<13, double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  sd)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(newton_group_kernel<13, float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  sf)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(newton_group_kernel<13, double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  sd)) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(newton_group_kernel<13, float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sf);
}

bool newton_supported(int nspec, int topo) {
    if (newton_group_case(nspec, topo)) return true;
#define X(ns, tp) \
    if (nspec == ns && topo == tp) return true;
    SDC_NEWTON_CASES(X)
#undef X
    return false;
}

// 7-and-fewer-species kernels: static grid (0), persistent grid with a per-lane
// work queue (1) or a per-warp one (2), and for the 5- and 7-species chains a
// group of 4 lanes per zone as for 13 species (3); 13-species chain: 4 (0) or
// 2 (1) lanes per zone, or one zone per thread as for the smaller networks on
// a static grid (2), with a per-lane (3) or a per-warp (4) work queue
int newton_variants(int nspec, int topo) {
    if (newton_group_case(nspec, topo)) return 5;
    return newton_small_group_case(nspec, topo) ? 4 : 3;
}

// Variants a matrix type runs: the float-pair matrix (prec 2) exists for the
// alpha chain's one-zone-per-thread kernels only (not the lane groups).
bool newton_variant_ok(int nspec, int topo, int prec, int variant) {
    if (variant < 0 || variant >= newton_variants(nspec, topo)) return false;
    if (prec != 2) return true;
    if (topo != TOPO_CHAIN) return false;
    if (newton_group_case(nspec, topo)) return variant >= 2;
    return !(newton_small_group_case(nspec, topo) && variant == 3);
}

int newton_default_variant(int nspec, int topo, int prec) {
    for (int v = 0; v < newton_variants(nspec, topo); v++)
        if (newton_variant_ok(nspec, topo, prec, v)) return v;
    return 0;
}


template <int NS, int TOPO>
int queue_blocks_per_sm(int prec) {
    int per = 0;
    if (prec == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, newton_queue_kernel<NS, TOPO, double>, NEWTON_BLOCK,
                                                      newton_smem_bytes<NS, double>(NEWTON_BLOCK));
    else if (prec == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, newton_queue_kernel<NS, TOPO, float>, NEWTON_BLOCK,
                                                      newton_smem_bytes<NS, float>(NEWTON_BLOCK));
    else if constexpr (TOPO == TOPO_CHAIN)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, newton_queue_kernel<NS, TOPO, f2>, NEWTON_BLOCK,
                                                      newton_smem_bytes<NS, f2>(NEWTON_BLOCK));
    return per;
}

int newton_persistent_blocks(const NetParams& P, int prec) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
#define X(ns, tp) \
    if (P.nspec == ns && P.topo == tp) per = queue_blocks_per_sm<ns, tp>(prec);
    SDC_NEWTON_CASES(X)
#undef X
    if (per < 1) per = 1;
    return sms * per;
}

// The one-zone-per-thread kernels with matrix type MT: static grid (kind 0),
// persistent grid with a per-lane (1) or a per-warp (2) work queue.
template <int NS, int TOPO, typename MT>
cudaError_t launch_per_zone(int kind, unsigned grid, unsigned pgrid, const NetParams& P, const NewtonCfg& cfg,
                            long long N, int dim, const double* rhs, const double* guess, const double* Rpred,
                            double* Uout, double* Rout, const double* dt_dev, double dt_frac, double dtm_host,
                            int* zone_status, int* zone_iters, DevStats* stats, unsigned long long* queue,
                            cudaStream_t st) {
    const size_t sm = newton_smem_bytes<NS, MT>(NEWTON_BLOCK);
    if (kind == 2)
        newton_warpqueue_kernel<NS, TOPO, MT><<<pgrid, NEWTON_BLOCK, sm, st>>>(
            P, cfg, N, dim, rhs, guess, Rpred, Uout, Rout, dt_dev, dt_frac, dtm_host, zone_status, zone_iters, stats,
            queue);
    else if (kind == 1)
        newton_queue_kernel<NS, TOPO, MT><<<pgrid, NEWTON_BLOCK, sm, st>>>(
            P, cfg, N, dim, rhs, guess, Rpred, Uout, Rout, dt_dev, dt_frac, dtm_host, zone_status, zone_iters, stats,
            queue);
    else
        newton_kernel<NS, TOPO, MT><<<grid, NEWTON_BLOCK, sm, st>>>(P, cfg, N, dim, rhs, guess, Rpred, Uout, Rout,
                                                                    dt_dev, dt_frac, dtm_host, zone_status,
                                                                    zone_iters, stats);
    return cudaGetLastError();
}

// The float-pair matrix exists for the alpha chain's bordered form only.
template <int NS, int TOPO>
cudaError_t launch_per_zone_pair(int kind, unsigned grid, unsigned pgrid, const NetParams& P, const NewtonCfg& cfg,
                                 long long N, int dim, const double* rhs, const double* guess, const double* Rpred,
                                 double* Uout, double* Rout, const double* dt_dev, double dt_frac, double dtm_host,
                                 int* zone_status, int* zone_iters, DevStats* stats, unsigned long long* queue,
                                 cudaStream_t st) {
    if constexpr (TOPO == TOPO_CHAIN)
        return launch_per_zone<NS, TOPO, f2>(kind, grid, pgrid, P, cfg, N, dim, rhs, guess, Rpred, Uout, Rout, dt_dev,
                                             dt_frac, dtm_host, zone_status, zone_iters, stats, queue, st);
    else
        return cudaErrorInvalidValue;
}

cudaError_t launch_newton(const NetParams& P, const NewtonCfg& cfg, int prec, long long N, int dim,
                          const double* rhs, const double* guess, const double* Rpred, double* Uout, double* Rout,
                          const double* dt_dev, double dt_frac, double dtm_host, int* zone_status,
                          int* zone_iters, DevStats* stats, cudaStream_t st, int variant,
                          unsigned long long* queue, int persistent_blocks) {
    if (N <= 0) return cudaSuccess;
    if (!newton_variant_ok(P.nspec, P.topo, prec, variant)) return cudaErrorInvalidValue;
    if (newton_group_case(P.nspec, P.topo) && variant < 2) {
        const unsigned ggrid = (unsigned)((N + GROUP_ZONES - 1) / GROUP_ZONES);
#define SDC_GROUP_LAUNCH(MT, L)                                                                                    \
    newton_group_kernel<13, MT, L><<<ggrid, 32 * L, group_smem<13, MT>(), st>>>(                                   \
        P, cfg, N, dim, rhs, guess, Rpred, Uout, Rout, dt_dev, dt_frac, dtm_host, zone_status, zone_iters, stats)
        if (variant == 1) {
            if (prec == 0) SDC_GROUP_LAUNCH(double, 2);
            else SDC_GROUP_LAUNCH(float, 2);
        } else {
            if (prec == 0) SDC_GROUP_LAUNCH(double, 4);
            else SDC_GROUP_LAUNCH(float, 4);
        }
#undef SDC_GROUP_LAUNCH
        return cudaGetLastError();
    }
    if (variant == 3 && newton_small_group_case(P.nspec, P.topo)) {
        const unsigned ggrid = (unsigned)((N + GROUP_ZONES - 1) / GROUP_ZONES);
#define SDC_SMALL_GROUP_LAUNCH(NSV, MT)                                                                            \
    newton_group_kernel<NSV, MT, 4><<<ggrid, 128, group_smem<NSV, MT>(), st>>>(                                      \
        P, cfg, N, dim, rhs, guess, Rpred, Uout, Rout, dt_dev, dt_frac, dtm_host, zone_status, zone_iters, stats)
        if (P.nspec == 5) {
            if (prec == 0) SDC_SMALL_GROUP_LAUNCH(5, double);
            else SDC_SMALL_GROUP_LAUNCH(5, float);
        } else {
            if (prec == 0) SDC_SMALL_GROUP_LAUNCH(7, double);
            else SDC_SMALL_GROUP_LAUNCH(7, float);
        }
#undef SDC_SMALL_GROUP_LAUNCH
        return cudaGetLastError();
    }
    // one zone per thread; the 13-species chain numbers these variants from 2
    if (newton_group_case(P.nspec, P.topo)) variant -= 2;
    const unsigned grid = (unsigned)((N + NEWTON_BLOCK - 1) / NEWTON_BLOCK);
    const bool q = (variant == 1 || variant == 2) && queue != nullptr && persistent_blocks > 0;
    const unsigned pgrid = q ? (unsigned)(persistent_blocks < (long long)grid ? persistent_blocks : grid) : 0u;
    const int kind = !q ? 0 : (variant == 2 ? 2 : 1);
#define X(ns, tp)                                                                                          \
    if (P.nspec == ns && P.topo == tp) {                                                                   \
        if (prec == 0)                                                                                     \
            return launch_per_zone<ns, tp, double>(kind, grid, pgrid, P, cfg, N, dim, rhs, guess, Rpred, Uout, \
                                                   Rout, dt_dev, dt_frac, dtm_host, zone_status, zone_iters, \
                                                   stats, queue, st);                                      \
        if (prec == 1)                                                                                     \
            return launch_per_zone<ns, tp, float>(kind, grid, pgrid, P, cfg, N, dim, rhs, guess, Rpred, Uout, \
                                                  Rout, dt_dev, dt_frac, dtm_host, zone_status, zone_iters, \
                                                  stats, queue, st);                                       \
        return launch_per_zone_pair<ns, tp>(kind, grid, pgrid, P, cfg, N, dim, rhs, guess, Rpred, Uout, Rout, \
                                            dt_dev, dt_frac, dtm_host, zone_status, zone_iters, stats, queue, st); \
    }
    SDC_NEWTON_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_reaction_source(const NetParams& P, long long N, int dim, const double* U, double* R,
                                   cudaStream_t st, double* anchor) {
    if (N <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((N + NEWTON_BLOCK - 1) / NEWTON_BLOCK);
    if (newton_group_case(P.nspec, P.topo)) {
        reaction_source_kernel<13, TOPO_CHAIN><<<grid, NEWTON_BLOCK, 0, st>>>(P, N, dim, U, R, anchor);
        return cudaGetLastError();
    }
#define X(ns, tp)                                                                              \
    if (P.nspec == ns && P.topo == tp) {                                                       \
        reaction_source_kernel<ns, tp><<<grid, NEWTON_BLOCK, 0, st>>>(P, N, dim, U, R, anchor); \
        return cudaGetLastError();                                                             \
    }
    SDC_NEWTON_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace sdcd
