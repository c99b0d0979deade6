// sdc_launch.h -- internal launchers shared by the translation units of libsdc.
#pragma once
#include <cuda_runtime.h>

#include "sdc_dev.cuh"
#include "sdc_stencil.cuh"

namespace sdcd {

// Newton kernel support: chain topology for these species counts, the generic
// topology for the small ones.
bool newton_supported(int nspec, int topo);
bool stencil_supported(int dim, int nspec);
cudaError_t newton_prepare(int nspec, int topo);  // raise the dynamic shared-memory limit
void stencil_tile(int dim, int nspec, int t[3]);
size_t stencil_smem_bytes(int dim, int nspec);
cudaError_t stencil_prepare(int dim, int nspec);  // raise the dynamic shared-memory limit

// dtm = (dt_dev ? *dt_dev * dt_frac : dtm_host)
cudaError_t launch_newton(const NetParams& P, const NewtonCfg& cfg, int prec, long long N, int dim,
                          const double* rhs, const double* guess, double* Uout, double* Rout,
                          const double* dt_dev, double dt_frac, double dtm_host, int* zone_status,
                          int* zone_iters, DevStats* stats, cudaStream_t st);

cudaError_t launch_reaction_source(const NetParams& P, long long N, int dim, const double* U, double* R,
                                   cudaStream_t st);

cudaError_t launch_stencil(const NetParams& P, int dim, int limiter, long long Ntot, const BoxDev* boxes,
                           const TileDev* tiles, int ntiles, const double* U, double* A, int mode,
                           const RhsArgs& ra, cudaStream_t st);

}  // namespace sdcd
