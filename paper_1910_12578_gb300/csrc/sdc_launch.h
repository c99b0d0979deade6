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
int stencil_variants(int dim, int nspec);  // tile shapes available to the autotuner
int stencil_split_variant(int dim, int nspec);  // the direction-split passes' variant, or -1
void split_tile_shape(int D, int t[3]);          // zones of one tile of pass D along x, y, z
void stencil_tile(int dim, int nspec, int variant, int t[3]);
size_t stencil_smem_bytes(int dim, int nspec, int variant);
cudaError_t stencil_prepare(int dim, int nspec);  // raise the dynamic shared-memory limit

// dtm = (dt_dev ? *dt_dev * dt_frac : dtm_host)
// variant 0: one zone per thread on a static grid; 1: persistent grid of
// persistent_blocks fed by the zero-initialised device counter *queue, one
// zone per lane at a time (zones of uneven cost balance across lanes); 2: the
// same grid and counter, 32 neighbouring zones per warp at a time.  The
// 13-species group kernel: 4 lanes per zone (0) or 2 (1).
int newton_variants(int nspec, int topo);
bool newton_variant_ok(int nspec, int topo, int prec, int variant);
int newton_default_variant(int nspec, int topo, int prec);
bool newton_group_case(int nspec, int topo);  // the 13-species chain (a group of lanes per zone)
// Rpred: R^{m+1,(k)} of the sweep (the start is then the explicit predictor where
// admissible, the guess elsewhere), or nullptr (the start is the guess)
cudaError_t launch_newton(const NetParams& P, const NewtonCfg& cfg, int prec, long long N, int dim,
                          const double* rhs, const double* guess, const double* Rpred, double* Uout, double* Rout,
                          const double* dt_dev, double dt_frac, double dtm_host, int* zone_status,
                          int* zone_iters, DevStats* stats, cudaStream_t st, int variant = 0,
                          unsigned long long* queue = nullptr, int persistent_blocks = 0);
int newton_persistent_blocks(const NetParams& P, int prec);  // resident blocks x SMs

// anchor: where non-null (alpha chain), the step's rate anchors of NewtonCfg at U
cudaError_t launch_reaction_source(const NetParams& P, long long N, int dim, const double* U, double* R,
                                   cudaStream_t st, double* anchor = nullptr);

cudaError_t launch_stencil(const NetParams& P, int dim, int limiter, long long Ntot, const BoxDev* boxes,
                           const TileDev* tiles, int ntiles, const double* U, double* A, int mode,
                           const RhsArgs& ra, cudaStream_t st, int variant = 0);
// the direction-split passes (3D): tiles[D] / ntiles[D] of pass D; prim is a
// field-major [nvar][Ntot] buffer for the primitives
cudaError_t launch_stencil_split(const NetParams& P, int limiter, long long Ntot, const BoxDev* boxes,
                                 const TileDev* const* tiles, const int* ntiles, const double* U, double* prim,
                                 double* A, int mode, const RhsArgs& ra, cudaStream_t st);

}  // namespace sdcd
