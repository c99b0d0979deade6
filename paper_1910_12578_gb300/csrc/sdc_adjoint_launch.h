// sdc_adjoint_launch.h -- internal launchers of the adjoint kernels.
#pragma once
#include <cuda_runtime.h>

#include "sdc_dev.cuh"
#include "sdc_stencil.cuh"

namespace sdcd {

// arguments of the adjoint of one node's right-hand side
struct RhsAdjArgs {
    int nvar, dim, M, m;
    long long N;
    const double* rhsbar;
    double* Ubar_m;         // adjoint of U_m (of this iteration), or of U^n for m = 0
    double* Abar_new_m;     // adjoint of A_m of this iteration (NULL for m = 0)
    double* Abar_old[MAXM];  // adjoints of A_l of the previous iteration
    double* Rbar_old[MAXM];  // adjoints of R_l of the previous iteration
    double dtm;
    double qdt[MAXM];        // q_{m,l} dt
};

bool adjoint_supported(int dim, int nspec, int topo);
cudaError_t launch_stencil_vjp(const NetParams& P, int dim, int limiter, long long N, const BoxDev* boxes, int nbox,
                               const double* U, const double* Abar, double* G, double* Ubar, cudaStream_t st,
                               int mode = 0);  // 0: reverse sweep per face, 1: forward-mode dual numbers
cudaError_t launch_reaction_vjp(const NetParams& P, int dim, long long N, const double* U, const double* Rbar,
                                double* Ubar, double dtm, double* rhsbar, double* abar_zone, cudaStream_t st);
cudaError_t launch_rhs_adjoint(const RhsAdjArgs& a, cudaStream_t st);
cudaError_t launch_reduce_rows(long long N, int rows, const double* x, double* out, cudaStream_t st);

}  // namespace sdcd
