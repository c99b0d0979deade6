// sdc_fourth_launch.h -- launchers of the fourth-order finite-volume operators
// (paper section 2: the fourth-order method pairs Simpson's rule with the
// spatial reconstruction of McCorquodale & Colella), smooth-flow form
// (limiter 0) or limited form (limiter 1: face averages limited per side,
// HLLC between the two sides).
#pragma once
#include <cuda_runtime.h>

#include "sdc_dev.cuh"
#include "sdc_stencil.cuh"

namespace sdcd {

// device workspace of the fourth-order operators (owned by the context)
struct FourthWs {
    double *Uc = nullptr, *W2 = nullptr, *Wc = nullptr, *Wa = nullptr;  // [nvar][N]
    double *Wf = nullptr, *Wfc = nullptr, *Fc = nullptr, *F2 = nullptr, *Fa = nullptr;  // smooth form: Wf, Wfc
    double *WL = nullptr, *WR = nullptr;  // limited form: the two sides of every face
    double *rc = nullptr, *gc = nullptr;  // zone-centre rhs and guess of the implicit update [nvar][N]
    double* Rc = nullptr;                 // zone-centre source [nspec + 1][N]
};

// kernel launches of one fourth-order advective term
inline int fourth_advective_launches(int dim, int limiter) { return 2 + (limiter ? 4 : 5) * dim; }
// kernel launches of one fourth-order implicit update (both maps, Newton, map and update)
constexpr int FOURTH_NEWTON_LAUNCHES = 3;
constexpr int FOURTH_SOURCE_LAUNCHES = 3;

// A = fourth-order advective term of the averages U (limiter: 0 smooth form, 1 limited form)
cudaError_t launch_advective4(const NetParams& P, int dim, int limiter, long long N, const BoxDev* boxes, int nbox,
                              const double* U, double* A, const FourthWs& w, cudaStream_t st);
// R = averaged reactive source, R(U_c) + L R(U_c)/24 with U_c = U - L U/24
cudaError_t launch_reaction_source4(const NetParams& P, int dim, long long N, const BoxDev* boxes, int nbox,
                                    const double* U, double* R, const FourthWs& w, cudaStream_t st);
// implicit update of the averages: solve at zone centres, then <U> = <rhs> + dt_m <R>
cudaError_t launch_newton4(const NetParams& P, const NewtonCfg& cfg, int prec, int dim, long long N,
                           const BoxDev* boxes, int nbox, const double* rhs, const double* guess, double* Uout,
                           double* Rout, const double* dt_dev, double dt_frac, double dtm_host, int* zone_status,
                           int* zone_iters, DevStats* stats, const FourthWs& w, cudaStream_t st, int variant,
                           unsigned long long* queue, int persistent_blocks);

}  // namespace sdcd
