/*
 * sdc.h -- C ABI of libsdc: the data-parallel hot path of the spectral
 * deferred correction (SDC) coupling of hydrodynamics and reactions of
 * arXiv:1910.12578 (Castro), section 2, on one NVIDIA GB300 (sm_103a).
 *
 * The method (section 2):
 *   Eq. 1            U_t = A(U) + R(U): A is the divergence of the
 *                    hydrodynamic fluxes, R the reactive sources.
 *   Eq. sdc:general  from temporal node m to m+1, iteration k -> k+1,
 *     U^{m+1,(k+1)} = U^{m,(k+1)} + dt_m [A^{m,(k+1)} - A^{m,(k)}]
 *                   + dt_m [R^{m+1,(k+1)} - R^{m+1,(k)}]
 *                   + int_{t^m}^{t^{m+1}} (A^{(k)} + R^{(k)}) dt
 *   with zone averages, explicit in A and implicit in R (the new node state
 *   solves a nonlinear system zone by zone), the integral formed from the
 *   previous iterate at every node: trapezoid rule (2 Gauss-Lobatto nodes),
 *   Simpson's rule (3 Gauss-Lobatto nodes), or through the Radau points.
 *
 * Conventions used by every call:
 *   - Conserved fields, in this order: rho, rho*u_0..rho*u_{dim-1}, rho*E,
 *     rho*X_0..rho*X_{nspec-1};  nvar = 2 + dim + nspec.
 *   - Reactive fields (the unknowns of the implicit update and the layout of
 *     every R array): rho*E, rho*X_0..rho*X_{nspec-1};  n = nspec + 1.
 *   - Arrays are FP64, field-major and x fastest.  Several boxes are
 *     concatenated in the order given to sdc_init_box:
 *         U[f * Ntot + off_b + i + n0*(j + n1*k)],  Ntot = sum of box zones.
 *   - Every box is periodic on itself; its 2-zone halo is formed on chip
 *     from its own interior (no ghost storage in memory).
 *   - All array arguments are DEVICE pointers owned by the caller, 16-byte
 *     aligned.  The library owns only its workspace (inside the context).
 *   - Work is enqueued on the CUDA stream given to sdc_init_box (borrowed,
 *     not owned).  Calls that return host-visible results (stats, dt) wait
 *     for that stream; the others return after enqueueing.
 *   - Every call returns a status and never aborts, traps or exits.
 *   - Not thread safe per context; one GPU (the current device at
 *     sdc_init_box) per context.
 */
#ifndef SDC_H
#define SDC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdc_ctx sdc_ctx; /* opaque, owned by the library */

typedef enum {
    SDC_OK = 0,
    SDC_ERR_INVALID_ARG = 1,   /* a bad size, pointer, network or parameter */
    SDC_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
    SDC_ERR_OOM = 3,           /* workspace allocation failed */
    SDC_ERR_NEWTON_NOCONV = 4, /* some zones did not converge (best iterate kept) */
    SDC_ERR_NONPHYSICAL = 5,   /* a zone had no admissible Newton step */
    SDC_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
    SDC_ERR_TOO_LARGE = 7      /* the problem does not fit the fixed scratch of sdc_step_static */
} sdc_status;

/* Precision of the Newton matrix and its elimination (section 2's implicit
   reaction update; the residual, the rates, the quadrature and the update are
   FP64 in every mode):
   SDC_PREC_FP64       FP64 throughout;
   SDC_PREC_FP32_JAC   the Jacobian build and LU in FP32, so that Newton acts as
                       iterative refinement of the FP64 residual;
   SDC_PREC_FP32X2_JAC the Jacobian build and LU in pairs of FP32 values
                       (double-float arithmetic on the FP32 pipe, about 48
                       significant bits): Newton's step to about 2^-44 relative.
                       Alpha-chain networks only (SDC_ERR_INVALID_ARG otherwise),
                       one zone per thread (Newton variants without lane groups).
   The FP64 and FP32-pair modes start each node's Newton solve from the explicit
   predictor rhs + dt_m R^{m+1,(k)}; the FP32 mode from the previous iterate. */
typedef enum { SDC_PREC_FP64 = 0, SDC_PREC_FP32_JAC = 1, SDC_PREC_FP32X2_JAC = 2 } sdc_precision;

/* rate laws of the network: r_j = a_j rho^(o_j-1) f_j(T) prod_reactants Y^cnt,
   Y_i = X_i / mass_i, o_j = total reactant count */
enum { SDC_RATE_POWER = 0 /* f = T^nu */, SDC_RATE_ARRHENIUS = 1 /* f = exp(-nu/T) */ };

/* per-zone Newton outcome (zone_status arrays) */
enum { SDC_ZONE_OK = 0, SDC_ZONE_MAXIT = 1, SDC_ZONE_NONPHYSICAL = 2, SDC_ZONE_SINGULAR = 3 };

#define SDC_MAX_SPEC 16
#define SDC_MAX_REAC 16

/* one periodic box: dim in {1,2,3}, zones per axis (unused axes = 1), widths */
typedef struct {
    int dim;
    int n[3];
    double dx[3];
} sdc_box;

/* reaction network (host pointers, copied by sdc_init_box).
   R(rho X_i) = rho mass_i sum_j s_ij r_j,  R(rho E) = rho sum_j Q_j r_j,
   s_ij = (prod_j == i) - (reactant multiplicities of i in reaction j). */
typedef struct {
    int nspec, nreac, rate_law;
    const double* mass;   /* [nspec] species mass numbers            */
    const double* a;      /* [nreac] rate prefactors                 */
    const double* nu;     /* [nreac] exponent (power) or activation  */
    const double* Q;      /* [nreac] energy released per unit rate   */
    const int* reac;      /* [2*nreac] reactant species, -1 = none    */
    const int* cnt;       /* [2*nreac] reactant multiplicities        */
    const int* prod;      /* [nreac] product species                  */
} sdc_network;

typedef struct {
    double gamma;          /* gamma-law gas, p = rho T                      */
    int n_nodes;           /* M: temporal nodes including node 0 (2 or 3;
                              Radau also 4)                                   */
    int n_iters;           /* K: SDC iterations per step, >= 1              */
    int limiter;           /* order 2: 1 = MC limited PLM, 0 = centred PLM;  */
                           /* order 4: 1 = limited, 0 = smooth-flow form     */
    sdc_precision prec;    /* Newton linear algebra precision               */
    double newton_rtol;    /* scaled Newton update that ends the solve      */
    int newton_maxit;      /* iteration cap per zone solve                  */
    int node_type;         /* SDC_NODES_LOBATTO or SDC_NODES_RADAU          */
    int space_order;       /* 2: PLM + limiter + HLLC, R on zone averages;   */
                           /* 4: the fourth-order finite-volume operators    */
} sdc_params;

/* space_order = 4 (section 2: the fourth-order method pairs Simpson's rule with
   McCorquodale & Colella's reconstruction): zone centres f_c = <f> - L<f>/24
   (L: second differences summed over the dimensions), primitive averages
   W(U_c) + L W(<U>)/24, face averages by the 7/12, -1/12 stencil, face fluxes
   F_c + L_t F_2/24 (L_t: second differences across the face), averaged sources
   R(U_c) + L R(U_c)/24, and the implicit update solved at zone centres with
   <U> = <rhs> + dt_m <R>.  limiter = 0, smooth-flow form: F_c = F(W_f) at the
   face-centre state W_f = <W>_f - L_t <W>_f/24, F_2 = F(<W>_f), the physical
   flux.  limiter = 1, limited form: each face average is limited (Colella &
   Sekora's face limiter), every zone limits its two face values (a limited
   curvature at extrema, where a difference of averages within 2^-20 of the
   other side's or 2^-48 of the averages counts as a tie; the PPM overshoot
   bounds elsewhere) with the mass fractions
   renormalised, and F_c, F_2 are HLLC fluxes between the two limited sides (at
   the face centres, each side less L_t/24 of itself, and at the face averages).
   The adjoint and sdc_step_static take space_order 2 only. */

/* Temporal node sets of the SDC step (n_nodes = M):
   SDC_NODES_LOBATTO: Gauss-Lobatto nodes {0,1} or {0,1/2,1}; the integral of
     Eq. sdc:general by the trapezoid (M = 2) or Simpson's (M = 3) rule through
     all nodes (section 2).
   SDC_NODES_RADAU: node 0 at t^n and the M-1 right-endpoint Gauss-Radau points
     ({1}, {1/3, 1} or {(4-sqrt 6)/10, (4+sqrt 6)/10, 1}); the integral through
     those points only, so that the
     iteration converges to Radau IIA collocation, which is L-stable: an
     instance of the alternative quadratures for very stiff burning that the
     paper's closing section (Future Developments) names as work in progress. */
enum { SDC_NODES_LOBATTO = 0, SDC_NODES_RADAU = 1 };

typedef struct {
    long long newton_iters_total; /* sum over zone solves of the iterations   */
    long long newton_solves;      /* zone solves                              */
    long long n_fail;             /* zone solves not converged                */
    long long hist[64];           /* hist[i]: solves with i iterations (63 = 63+) */
} sdc_stats;

/* Create a context for nbox boxes with one network and one parameter set,
   allocate its device workspace and upload the network.
   Errors: SDC_ERR_INVALID_ARG (nbox < 1, bad dims, a box of 2^31 zones or
   more, nspec > SDC_MAX_SPEC, nreac > SDC_MAX_REAC, species index out of
   range, n_nodes not 2/3 (2-4 for Radau nodes), n_iters < 1, gamma <= 1,
   node_type or space_order not one of theirs), SDC_ERR_OOM, SDC_ERR_CUDA.
   *out is NULL on error. */
sdc_status sdc_init_box(const sdc_box* boxes, int nbox, const sdc_network* net,
                        const sdc_params* prm, void* cuda_stream, sdc_ctx** out);

/* A(U): advective term, the divergence of the HLLC fluxes of a method-of-lines
   PLM reconstruction (MC limiter) of the primitive variables
   (paper section 2, Eq. 1: A is minus the divergence of the advective fluxes).
   U, A: [nvar][Ntot] device arrays; A may not alias U. */
sdc_status sdc_advective_term(sdc_ctx* ctx, const double* U, double* A);

/* Node-to-node integral of Eq. sdc:general from node m to m+1 (0 <= m < M-1):
   I = sum_l q_{m,l} dt (A_l + R_l), q the trapezoid / Simpson weights.
   A_nodes: [M][nvar][Ntot], R_nodes: [M][n][Ntot] (R enters the reactive
   fields only), I: [nvar][Ntot]. */
sdc_status sdc_node_integral(sdc_ctx* ctx, const double* A_nodes, const double* R_nodes,
                             double dt, int m, double* I);

/* Implicit reaction update of Eq. sdc:general at every zone:
   solve  w - dt_m R(w; rho, rho u) = rhs_w  for the reactive fields w, with
   rho and rho*u taken from rhs (R has no mass or momentum component), by
   Newton iteration on the analytic Jacobian I - dt_m dR/dw globalised by
   pseudo-transient continuation.  The linear systems: dense LU with partial
   pivoting for a general network; for the alpha chain, elimination of its
   bordered bidiagonal form (chain species first, pivoting within the band,
   then the 2 x 2 alpha / energy block), the same solution to rounding.
   rhs: [nvar][Ntot].  U_inout: [nvar][Ntot], the guess on entry (its mass
   fractions and specific energy are carried to the density of rhs), the
   solution on exit.  R_out: [n][Ntot] = R(solution).  zone_status, zone_iters:
   [Ntot] or NULL.  stats: NULL (asynchronous) or filled after a wait.
   Returns SDC_ERR_NEWTON_NOCONV when stats is given and some zone failed. */
sdc_status sdc_react_newton(sdc_ctx* ctx, const double* rhs, double dt_m, double* U_inout,
                            double* R_out, int* zone_status, int* zone_iters, sdc_stats* stats);

/* One SDC time step of size dt, in place on U ([nvar][Ntot]): every node starts
   at U^n, then K iterations of the node-to-node sweep of Eq. sdc:general;
   U^{n+1} = U^{M-1,(K)}.  Replays a CUDA graph captured at the first call for
   this U pointer (the graphs of the last two U pointers are kept, so a caller
   that alternates two buffers replays both).  stats: NULL (asynchronous) or
   filled after a wait;
   returns SDC_ERR_NEWTON_NOCONV when stats is given and some zone failed. */
sdc_status sdc_step(sdc_ctx* ctx, double* U, double dt, sdc_stats* stats);

/* Per-class CUDA-event times of one eagerly launched step. */
typedef struct {
    int launches_stencil, launches_newton, launches_other;
    float ms_stencil, ms_newton, ms_other; /* summed event durations of those launches */
} sdc_profile;

/* sdc_step without the graph: the same kernels with the same arguments (same
   results), each launch bracketed by CUDA events on the context stream, for
   measurement.  Waits for the stream.  stats as in sdc_step. */
sdc_status sdc_step_profile(sdc_ctx* ctx, double* U, double dt, sdc_stats* stats, sdc_profile* prof);

/* Diagnostic: the library's refined reciprocal and square root (used
   inside its kernels in place of IEEE division and sqrt) for n positive normal
   doubles x (device arrays), for testing against correctly rounded results. */
sdc_status sdc_selftest_math(const double* x, long long n, double* rcp_out, double* sqrt_out, void* cuda_stream);

/* Diagnostic: the library's power-law rate factor T^nu = 2^(nu log2 T) (its
   table-driven log2 and exp2, used by the reaction kernels in place of
   exp(nu log T)) for n pairs (T, nu) of device doubles, T > 0; out[i] = T[i]^nu[i].
   Asynchronous on cuda_stream. */
sdc_status sdc_selftest_pow(const double* T, const double* nu, long long n, double* out, void* cuda_stream);

/* Kernel variants of a context, chosen by measurement.
   stencil: tile shape of the advective-term kernel (0: 8^3 zones, 576 threads,
   one face per thread per direction; 1: 8 x 8 x 4 zones, 320 threads; one shape
   only in 1D and for 13 species).  newton, networks of up to 7 species: 0 = one
   zone per thread on a static grid; 1 = a persistent grid fed by a device work
   queue, each lane taking the next zone when its own is solved, so zones with
   many Newton iterations do not hold their warp; 2 = the same with a queue of
   32-zone chunks per warp; 3 (5- and 7-species chains) = a group of 4 lanes per
   zone.  13-species chain: 0 / 1 = a group of 4 / 2 lanes per zone; 2, 3, 4 =
   variants 0, 1, 2 of the smaller networks.  Defaults: 0, 0 (SDC_PREC_FP32X2_JAC,
   which has no lane-group kernels: Newton default 2 for 13 species; variant 3
   of the smaller chains and 0, 1 of the 13-species chain are refused by
   sdc_set_variants and skipped by sdc_autotune, whose ms_newton stays 0 there). */
#define SDC_MAX_VARIANTS 8
typedef struct {
    int stencil_variants, newton_variants;  /* candidates tried */
    int stencil_choice, newton_choice;      /* chosen */
    float ms_stencil[SDC_MAX_VARIANTS], ms_newton[SDC_MAX_VARIANTS];  /* per candidate: event time of one step */
} sdc_tuning;

/* Time one eager step per candidate on a scratch copy of U (U is not changed)
   and keep the fastest tile shape and Newton variant for the context; the next
   sdc_step recaptures its graph.  Allocates and frees one U-sized scratch
   array; waits for the stream.  out may be NULL. */
sdc_status sdc_autotune(sdc_ctx* ctx, const double* U, double dt, sdc_tuning* out);

/* Set the variants directly (as sdc_autotune would). */
sdc_status sdc_set_variants(sdc_ctx* ctx, int stencil_variant, int newton_variant);

/* Number of kernels one sdc_step launches (its graph plus the dt store). */
sdc_status sdc_launches_per_step(const sdc_ctx* ctx, int* launches);

/* Adjoint of one SDC step (vector-Jacobian product of sdc_step):
     gU_n = (dU^{n+1}/dU^n)^T gU_np1,   g_a += (dU^{n+1}/da)^T gU_np1
   with a the rate prefactors of the network.  U_n is the step's checkpoint
   (its input state); the step is recomputed from it with every node state kept,
   then swept in reverse: the implicit reaction update through the
   implicit-function theorem (a transposed solve with the Jacobian at the
   converged root), the right-hand side and quadrature as linear maps, and the
   advective term through its face fluxes with the limiter and HLLC branches of
   the recomputed step fixed.  All pointers are device arrays: U_n, gU_np1, gU_n
   [nvar][Ntot]; g_a [nreac], accumulated (NULL: not formed).  The first call
   allocates an adjoint workspace in the context (for 3 nodes and K
   iterations about (13 + 2K) nvar + 7 (nspec+1) + 12 nvar + nreac doubles per
   zone).  Supported: the A -> B network in 1D and 3D and the 5-, 7- and
   13-species alpha chains in 3D (the chains' transposed solve by the bordered
   chain elimination, in reversed chain order), second-order operators:
   SDC_ERR_INVALID_ARG otherwise.  Deterministic (no floating-point atomics). */
sdc_status sdc_step_backward(sdc_ctx* ctx, const double* U_n, double dt, const double* gU_np1, double* gU_n,
                             double* g_a);

/* Strang-split baseline step (no counterpart in the method itself: section 2
   contrasts the SDC update with operator splitting, whose coupling error the
   SDC update removes): reactions over dt/2, advection over dt, reactions over
   dt/2, each sub-problem integrated by this context's SDC step (same nodes,
   iterations, kernels and precision) with the other operator set to zero; with
   R = 0 the implicit update is w = rhs.  U: device [nvar][Ntot], advanced in
   place.  stats as in sdc_step (summed over the two reaction sub-steps).  The
   three sub-steps are captured as one CUDA graph per U pointer. */
sdc_status sdc_step_strang(sdc_ctx* ctx, double* U, double dt, sdc_stats* stats);

/* Vector-Jacobian product of the advective term A(U) of Eq. 1 (section 2: minus
   the divergence of the advective fluxes):  Ubar += (dA/dU)^T Abar  at the state
   U, with the branches of the MC limiter and of HLLC those that U selects.
   U, Abar, Ubar: device arrays [nvar][Ntot]; Ubar is accumulated.  mode 0: a
   reverse sweep through each face flux (what sdc_step_backward uses); mode 1:
   forward-mode dual numbers, one input direction at a time (4 nvar passes per
   face: an independent formulation, slower, for cross-checks).  Both write
   per-face products to the adjoint workspace (allocated on first use) and add
   them up per zone in a fixed order (deterministic).  Supported networks as in
   sdc_step_backward; SDC_ERR_INVALID_ARG otherwise or for another mode.
   Asynchronous on the context's stream. */
sdc_status sdc_advective_term_vjp(sdc_ctx* ctx, const double* U, const double* Abar, double* Ubar, int mode);

/* Replace the rate prefactors a_j of the context's network (host array [nreac]). */
sdc_status sdc_set_rates(sdc_ctx* ctx, const double* a);

/* CFL time step: dt = cfl / max over zones of sum_d (|u_d| + c) / dx_d.
   Waits for the stream; *dt_out is a host pointer. */
sdc_status sdc_cfl_dt(sdc_ctx* ctx, const double* U, double cfl, double* dt_out);

/* Sizes of the context: total zones, nvar, n (reactive fields). */
sdc_status sdc_sizes(const sdc_ctx* ctx, long long* ntot, int* nvar, int* nreactive);

/* One SDC step that allocates nothing (the paper has no counterpart: this is a
   convenience of this library).  It is meant for callers that cannot call
   cudaMalloc: code running under an allocator or memory budget that another
   framework owns, hosts that forbid device allocations after start-up, or
   code that must not trigger the implicit synchronisation of an allocation.
   Same arguments and results as sdc_init_box + sdc_step + sdc_destroy (the
   same kernels, launched eagerly on cuda_stream), but the whole workspace
   (node states, A and R of two iterations, the rhs, box and tile tables, dt,
   statistics) lives in one file-scope device array of SDC_STATIC_SCRATCH_BYTES
   that every GPU loading the library holds until the process exits.
   - Capacity: (2 + 3(M-1))*nvar + (1 + 2(M-1))*n doubles per zone (n = nspec
     + 1; each array rounded up to 256 bytes) plus the box and tile tables must
     fit in SDC_STATIC_SCRATCH_BYTES (48 MiB: e.g. 32^3 zones with 7 species
     and 3 nodes, 136 doubles per zone); larger problems, and boxes of 2^31
     zones or more, return SDC_ERR_TOO_LARGE before any work is enqueued; at
     most SDC_STATIC_MAX_BOXES boxes.
   - The first call on a device looks up the array's device address with
     cudaGetSymbolAddress (that device current); make that first call before
     any stream capture.
   - All calls share the array and it keeps the last call's contents (the
     statistics are cleared by every call).  Calls whose work overlaps on the
     GPU (other streams, other threads) race on it: serialise them.
   - stats: NULL (asynchronous) or filled after waiting for cuda_stream;
     SDC_ERR_NEWTON_NOCONV as in sdc_step.
   It calls no cudaMalloc, cudaFree or other allocating routine.  n_nodes 2 or 3
   (four Radau nodes need a context). */
#define SDC_STATIC_SCRATCH_BYTES (48ull << 20)
#define SDC_STATIC_MAX_BOXES 32
sdc_status sdc_step_static(const sdc_box* boxes, int nbox, const sdc_network* net, const sdc_params* prm,
                           void* cuda_stream, double* U, double dt, sdc_stats* stats);

/* Release the context and its workspace (NULL is allowed). */
void sdc_destroy(sdc_ctx* ctx);

/* Static description of a status code. */
const char* sdc_status_string(sdc_status s);

#ifdef __cplusplus
}
#endif
#endif /* SDC_H */
