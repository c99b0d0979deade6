/*
 * sdc_oracle.h -- plain FP64 CPU oracle of the SDC hydro + reaction sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library and its Python binding) never calls it and shares no
 * source with it.
 *
 * What it computes (paper section 2):
 *   U_t = A(U) + R(U)                                      (Eq. 1)
 *   U^{m+1,(k+1)} = U^{m,(k+1)} + dt_m [A^{m,(k+1)} - A^{m,(k)}]
 *                 + dt_m [R^{m+1,(k+1)} - R^{m+1,(k)}]
 *                 + int_{t^m}^{t^{m+1}} (A^{(k)} + R^{(k)}) dt   (Eq. sdc:general)
 * with zone averages, R evaluated on the zone average, the nonlinear system of
 * the new node state solved by Newton iteration, and the integral formed from
 * the previous iterate at every node (trapezoid rule for 2 nodes, Simpson's
 * rule for 3 nodes; or through the Radau points).
 *
 * Conventions (shared by every function here):
 *   dim in {1,2,3}; nvar = 2 + dim + nspec;
 *   conserved field order [rho, rho*u_0..rho*u_{dim-1}, rho*E, rho*X_0..rho*X_{nspec-1}];
 *   arrays are field-major, x fastest: U[f*N + i + n0*(j + n1*k)], N = n0*n1*n2;
 *   every box is periodic on itself;
 *   the reactive unknowns are the n = nspec+1 contiguous fields starting at
 *   rho*E, so reactive arrays R[r*N + zone] hold r = 0 -> rho*E, r = 1+i -> rho*X_i.
 */
#ifndef SDC_ORACLE_H
#define SDC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_SPEC 32
#define ORC_MAX_REAC 32

/* rate laws: r_j = a_j rho^(o_j-1) f_j(T) prod_reactants Y^count */
#define ORC_RATE_POWER 0      /* f = T^nu                   */
#define ORC_RATE_ARRHENIUS 1  /* f = exp(-nu / T)           */

/* per-zone Newton outcome */
#define ORC_NEWTON_OK 0
#define ORC_NEWTON_MAXIT 1
#define ORC_NEWTON_NONPHYSICAL 2
#define ORC_NEWTON_SINGULAR 3

typedef struct {
    int dim;            /* 1, 2 or 3                                       */
    int n[3];           /* zones per axis (unused axes = 1)                */
    double dx[3];       /* zone widths                                     */
    double gamma;       /* gamma-law gas                                   */
    int limiter;        /* 1 = MC limited PLM, 0 = unlimited centred PLM   */
    int nspec, nreac, rate_law;
    double mass[ORC_MAX_SPEC];          /* species mass numbers          */
    double a[ORC_MAX_REAC], nu[ORC_MAX_REAC], Q[ORC_MAX_REAC];
    int reac[ORC_MAX_REAC][2];          /* reactant species, -1 = none   */
    int cnt[ORC_MAX_REAC][2];           /* reactant multiplicities        */
    int prod[ORC_MAX_REAC];             /* product species                */
    int n_nodes;        /* M: temporal nodes including node 0 at t^n       */
    int n_iters;        /* K: SDC iterations per step                      */
    double newton_rtol; /* scaled update norm that ends the Newton loop    */
    int newton_maxit;
    int node_type;      /* ORC_NODES_LOBATTO (M = 2: trapezoid, 3: Simpson)  */
                        /* or ORC_NODES_RADAU (M = 2..4: Radau IIA points)   */
    int split_op;       /* ORC_OP_BOTH (the coupled SDC step), ORC_OP_ADVECT  */
                        /* (R = 0) or ORC_OP_REACT (A = 0): the sub-problems  */
                        /* of the Strang-split baseline                       */
    int space_order;    /* 2: PLM/HLLC, R on zone averages; 4: the fourth-    */
                        /* order operators (orc_advective4, ..._newton4)      */
} orc_problem;

#define ORC_OP_BOTH 0
#define ORC_OP_ADVECT 1
#define ORC_OP_REACT 2

#define ORC_NODES_LOBATTO 0
#define ORC_NODES_RADAU 1

typedef struct {
    long long newton_iters_total;
    long long newton_solves;
    long long n_fail;
    long long hist[64];  /* hist[i] = zones that took i iterations (i capped at 63) */
} orc_stats;

/* number of conserved fields */
int orc_nvar(const orc_problem* P);

/* node positions in [0,1] and node-to-node weights q[m*M + l] (units of dt),
   q_{m,l} = int_{tau_m}^{tau_{m+1}} L_l(tau) dtau (L_l through the interpolation
   nodes of the node type).  Returns 0 or -1 for a bad type or M. */
int orc_nodes(int type, int M, double* tau);
int orc_quad_weights(int type, int M, double* q);

/* ideal-gas helpers at one zone (conserved in, primitive out) */
double orc_temperature(const orc_problem* P, double rho, const double* mom, double rhoE);

/* advective term A(U) = -div F, MOL PLM + limiter + HLLC, periodic box */
void orc_advective(const orc_problem* P, const double* U, double* A);

/* HLLC flux through one face, primitive states q = [rho, u_0.., p, X_0..] (nvar entries) */
void orc_hllc(const orc_problem* P, int dir, const double* qL, const double* qR, double* F);

/* the HLLC fan of one face: wave speeds S[3] = {S_L, S*, S_R} and the star
   states U*_L, U*_R (2 + dim conserved entries: mass, momenta, energy) */
void orc_hllc_star(const orc_problem* P, int dir, const double* qL, const double* qR, double* S, double* UsL,
                   double* UsR);

/* reactive source R(w) (n entries) and dR/dw (n*n, row major) at one zone */
void orc_rates(const orc_problem* P, double rho, const double* mom, const double* w,
               double* R, double* dRdw /* nullable */);

/* reactive source for every zone of U: R[r*N + zone] */
void orc_reaction_source(const orc_problem* P, const double* U, double* R);

/* Newton solve of w - dt_m R(w) = rhs_w at one zone; w holds the guess on entry
   and the last iterate on exit.  Returns an ORC_NEWTON_* code; *iters gets the count. */
int orc_newton_zone(const orc_problem* P, double rho, const double* mom, const double* rhs_w,
                    double dt_m, double* w, int* iters);

/* implicit reaction update for every zone.  rhs: nvar*N.  U_inout: nvar*N guess in,
   solution out (rho and momenta copied from rhs).  R_out: n*N = R(solution).
   zone_status / zone_iters nullable. */
void orc_react_newton(const orc_problem* P, const double* rhs, double dt_m, double* U_inout,
                      double* R_out, int* zone_status, int* zone_iters, orc_stats* st);

/* I_m = sum_l q_{m,l} (A_l + R_l) over the nodes (A: M arrays of nvar*N, R: M arrays of n*N);
   I: nvar*N, zero in rho and momenta apart from the A part */
void orc_node_integral(const orc_problem* P, const double* const* A_nodes,
                       const double* const* R_nodes, double dt, int m, double* I);

/* one SDC time step of size dt, in place on U (nvar*N) */
int orc_sdc_step(const orc_problem* P, double* U, double dt, orc_stats* st);

/* Fourth-order operators (space_order = 4): average <-> zone-centre maps
   over nf field-major fields, the advective term, the averaged reactive
   source and the implicit update solved at zone centres. */
void orc_avg_to_point(const orc_problem* P, int nf, const double* avg, double* point);
void orc_point_to_avg(const orc_problem* P, int nf, const double* point, double* avg);
void orc_advective4(const orc_problem* P, const double* U, double* A);
/* the limited left (WL: upper face of zone z) and right (WR at z: lower face of
   zone z+1) states of direction dir from averaged primitives Wa and face values
   Wf, all [nvar][N] (the fourth-order form's limiters) */
void orc_limited_faces(const orc_problem* P, int dir, const double* Wa, const double* Wf, double* WL, double* WR);
void orc_advective_term(const orc_problem* P, const double* U, double* A);
void orc_reaction_source4(const orc_problem* P, const double* U, double* R);
void orc_react_newton4(const orc_problem* P, const double* rhs, double dt_m, double* U_inout, double* R_out,
                       orc_stats* st);

/* Strang-split baseline (section 2 contrasts SDC with operator splitting,
   whose coupling error SDC removes): reactions over dt/2, advection over dt,
   reactions over dt/2, each sub-problem integrated by the SDC step of P with
   the other operator set to zero.  Returns 0 or -1. */
int orc_strang_step(const orc_problem* P, double* U, double dt, orc_stats* st);

/* dt = cfl / max_zones sum_d (|u_d| + c) / dx_d */
double orc_cfl_dt(const orc_problem* P, const double* U, double cfl);

/* sweep control exposed for the tests: one SDC step where the caller also
   receives the final node states (M*nvar*N) */
int orc_sdc_step_nodes(const orc_problem* P, double* U, double dt, orc_stats* st, double* nodes_out);

#ifdef __cplusplus
}
#endif
#endif
