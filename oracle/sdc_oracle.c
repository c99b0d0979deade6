/*
 * sdc_oracle.c -- plain FP64 CPU oracle of the SDC hydro + reaction sweep.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline of the
 * benchmark).  Written to be read against the paper, not to be fast:
 * straight loops, no blocking, no fusion, compiled with -ffp-contract=off.
 *
 * Section map of the paper (arXiv:1910.12578):
 *   Eq. 1 (section 2)          U_t = A(U) + R(U)                 -> orc_sdc_step
 *   Eq. sdc:general (sec. 2)   node-to-node correction update    -> sdc_sweep_node
 *   section 2, after the eq.   zone averages, implicit in the new state,
 *                              integral from iteration (k) at all nodes,
 *                              trapezoid (2 nodes) / Simpson (3 nodes)
 * The paper does not specify the spatial operator, the networks, the EOS or
 * the Newton solve.  Readings taken here: method-of-lines PLM with the MC
 * limiter (or unlimited centred slopes) and Toro's HLLC flux with Davis wave
 * speeds; interface mass fractions renormalised to sum to one and species
 * carried by the mass flux of the side upwind of the contact; a gamma-law gas
 * p = rho T; the alpha-chain and A -> B networks with rates
 * r_j = a_j rho^(o_j - 1) f_j(T) prod Y^count; all nodes of the first
 * iterate equal to U^n; the implicit update solved by Newton iteration with
 * pseudo-transient continuation and a dense partially pivoted LU.
 */
#include "sdc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(P, i, j, k) ((i) + (P)->n[0] * ((j) + (P)->n[1] * (k)))

int orc_nvar(const orc_problem* P) { return 2 + P->dim + P->nspec; }

static long long nzones(const orc_problem* P) {
    return (long long)P->n[0] * P->n[1] * P->n[2];
}

/* ------------------------------------------------------------------ */
/* Temporal nodes and the node-to-node quadrature (section 2: the     */
/* integral of Eq. sdc:general, trapezoid / Simpson rule).            */
/* Gauss-Lobatto nodes on [0,1]: M=2 -> {0,1}, M=3 -> {0,1/2,1}; the   */
/* quadrature interpolates through all M nodes.                       */
/* Radau (section 5, Future Developments: other quadratures for very  */
/* stiff burning):                                                     */
/* node 0 at t^n and the s = M-1 right-endpoint Gauss-Radau points,   */
/* the zeros of P_s(2t-1) - P_{s-1}(2t-1) (P Legendre): s=1 -> {1},   */
/* s=2 -> {1/3, 1}, s=3 -> {(4-sqrt6)/10, (4+sqrt6)/10, 1}; the        */
/* quadrature interpolates through those s points only, so that the   */
/* converged sweep is Radau IIA collocation.                          */
/* ------------------------------------------------------------------ */
int orc_nodes(int type, int M, double* tau) {
    if (type == ORC_NODES_LOBATTO) {
        if (M == 2) { tau[0] = 0.0; tau[1] = 1.0; return 0; }
        if (M == 3) { tau[0] = 0.0; tau[1] = 0.5; tau[2] = 1.0; return 0; }
        return -1;
    }
    if (type == ORC_NODES_RADAU) {
        tau[0] = 0.0;
        if (M == 2) { tau[1] = 1.0; return 0; }
        if (M == 3) { tau[1] = 1.0 / 3.0; tau[2] = 1.0; return 0; }
        if (M == 4) {
            tau[1] = (4.0 - sqrt(6.0)) / 10.0;
            tau[2] = (4.0 + sqrt(6.0)) / 10.0;
            tau[3] = 1.0;
            return 0;
        }
        return -1;
    }
    return -1;
}

/* q_{m,l} = integral over [tau_m, tau_{m+1}] of the Lagrange basis
   polynomial L_l through the interpolation nodes (all M for Lobatto, nodes
   1..M-1 for Radau; q_{m,0} = 0 there).  The polynomial is expanded into
   monomial coefficients and integrated term by term. */
int orc_quad_weights(int type, int M, double* q) {
    double tau[8];
    if (orc_nodes(type, M, tau) != 0) return -1;
    int l0 = (type == ORC_NODES_RADAU) ? 1 : 0;
    for (int m = 0; m < M - 1; m++) q[m * M + 0] = 0.0;
    for (int l = l0; l < M; l++) {
        /* coefficients c[0..] of L_l(t) = prod_{j!=l} (t - tau_j)/(tau_l - tau_j) */
        double c[8] = {0};
        c[0] = 1.0;
        int deg = 0;
        for (int j = l0; j < M; j++) {
            if (j == l) continue;
            double den = tau[l] - tau[j];
            double nc[8] = {0};
            for (int p = 0; p <= deg; p++) {
                nc[p + 1] += c[p] / den;
                nc[p] += -tau[j] * c[p] / den;
            }
            deg++;
            for (int p = 0; p <= deg; p++) c[p] = nc[p];
        }
        for (int m = 0; m < M - 1; m++) {
            double a = tau[m], b = tau[m + 1], s = 0.0;
            for (int p = 0; p <= deg; p++)
                s += c[p] * (pow(b, p + 1) - pow(a, p + 1)) / (p + 1);
            q[m * M + l] = s;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* gamma-law EOS: p = rho T (R/mu = 1), e = T/(gamma-1)               */
/* ------------------------------------------------------------------ */
double orc_temperature(const orc_problem* P, double rho, const double* mom, double rhoE) {
    double m2 = 0.0;
    for (int d = 0; d < P->dim; d++) m2 += mom[d] * mom[d];
    double rhoe = rhoE - 0.5 * m2 / rho;
    return (P->gamma - 1.0) * rhoe / rho;
}

/* conserved -> primitive q = [rho, u_0.., p, X_0..] at one zone */
static void cons_to_prim(const orc_problem* P, const double* U, long long N, long long z, double* q) {
    int dim = P->dim;
    double rho = U[0 * N + z];
    q[0] = rho;
    double ke = 0.0;
    for (int d = 0; d < dim; d++) {
        double u = U[(1 + d) * N + z] / rho;
        q[1 + d] = u;
        ke += 0.5 * rho * u * u;
    }
    double rhoE = U[(1 + dim) * N + z];
    q[1 + dim] = (P->gamma - 1.0) * (rhoE - ke);
    for (int s = 0; s < P->nspec; s++) q[2 + dim + s] = U[(2 + dim + s) * N + z] / rho;
}

/* ------------------------------------------------------------------ */
/* HLLC approximate Riemann solver (Toro), Davis wave-speed estimates. */
/* Species flux = X of the side upwind of the contact times mass flux. */
/* ------------------------------------------------------------------ */

/* Wave speeds S = {S_L, S*, S_R} and the two star states U*_L, U*_R (mass,
   momenta, energy: 2 + dim entries each) of the HLLC fan between the
   primitive states qL and qR.  Each star state follows from the jump
   conditions across its outer wave with the contact moving at S* and one
   pressure on both sides of it:
     rho*_K = rho_K (S_K - u_K) / (S_K - S*),  u*_K = S*, tangential u kept,
     E*_K = rho*_K (E_K/rho_K + (S* - u_K)(S* + p_K / (rho_K (S_K - u_K)))). */
void orc_hllc_star(const orc_problem* P, int dir, const double* qL, const double* qR, double* S, double* UsL,
                   double* UsR) {
    int dim = P->dim;
    double g = P->gamma;
    double rL = qL[0], rR = qR[0];
    double unL = qL[1 + dir], unR = qR[1 + dir];
    double pL = qL[1 + dim], pR = qR[1 + dim];
    double kL = 0.0, kR = 0.0;
    for (int d = 0; d < dim; d++) {
        kL += qL[1 + d] * qL[1 + d];
        kR += qR[1 + d] * qR[1 + d];
    }
    double EL = pL / (g - 1.0) + 0.5 * rL * kL;   /* total energy per volume */
    double ER = pR / (g - 1.0) + 0.5 * rR * kR;
    double cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);

    double SL = fmin(unL - cL, unR - cR);
    double SR = fmax(unL + cL, unR + cR);
    double Ss = (pR - pL + rL * unL * (SL - unL) - rR * unR * (SR - unR)) /
                (rL * (SL - unL) - rR * (SR - unR));
    S[0] = SL; S[1] = Ss; S[2] = SR;

    double fac = rL * (SL - unL) / (SL - Ss);
    UsL[0] = fac;
    for (int d = 0; d < dim; d++) UsL[1 + d] = fac * (d == dir ? Ss : qL[1 + d]);
    UsL[1 + dim] = fac * (EL / rL + (Ss - unL) * (Ss + pL / (rL * (SL - unL))));
    fac = rR * (SR - unR) / (SR - Ss);
    UsR[0] = fac;
    for (int d = 0; d < dim; d++) UsR[1 + d] = fac * (d == dir ? Ss : qR[1 + d]);
    UsR[1 + dim] = fac * (ER / rR + (Ss - unR) * (Ss + pR / (rR * (SR - unR))));
}

void orc_hllc(const orc_problem* P, int dir, const double* qL, const double* qR, double* F) {
    int dim = P->dim;
    double g = P->gamma;
    double rL = qL[0], rR = qR[0];
    double unL = qL[1 + dir], unR = qR[1 + dir];
    double pL = qL[1 + dim], pR = qR[1 + dim];
    double kL = 0.0, kR = 0.0;
    for (int d = 0; d < dim; d++) {
        kL += qL[1 + d] * qL[1 + d];
        kR += qR[1 + d] * qR[1 + d];
    }
    double EL = pL / (g - 1.0) + 0.5 * rL * kL;
    double ER = pR / (g - 1.0) + 0.5 * rR * kR;
    double S[3], UsL[8], UsR[8];
    orc_hllc_star(P, dir, qL, qR, S, UsL, UsR);
    double SL = S[0], Ss = S[1], SR = S[2];

    /* physical fluxes and conserved states of both sides (mass, momenta, energy) */
    double FL[8], FR[8], UL[8], UR[8];
    int nh = 2 + dim; /* rho, momenta, energy */
    UL[0] = rL; UR[0] = rR;
    FL[0] = rL * unL; FR[0] = rR * unR;
    for (int d = 0; d < dim; d++) {
        UL[1 + d] = rL * qL[1 + d];
        UR[1 + d] = rR * qR[1 + d];
        FL[1 + d] = rL * unL * qL[1 + d] + (d == dir ? pL : 0.0);
        FR[1 + d] = rR * unR * qR[1 + d] + (d == dir ? pR : 0.0);
    }
    UL[1 + dim] = EL; UR[1 + dim] = ER;
    FL[1 + dim] = (EL + pL) * unL;
    FR[1 + dim] = (ER + pR) * unR;

    /* the region of the fan that holds the face: F_L, F*_L = F_L + S_L (U*_L - U_L),
       F*_R = F_R + S_R (U*_R - U_R), F_R */
    double Fh[8];
    if (SL >= 0.0) {
        for (int f = 0; f < nh; f++) Fh[f] = FL[f];
    } else if (Ss >= 0.0) {
        for (int f = 0; f < nh; f++) Fh[f] = FL[f] + SL * (UsL[f] - UL[f]);
    } else if (SR > 0.0) {
        for (int f = 0; f < nh; f++) Fh[f] = FR[f] + SR * (UsR[f] - UR[f]);
    } else {
        for (int f = 0; f < nh; f++) Fh[f] = FR[f];
    }
    for (int f = 0; f < nh; f++) F[f] = Fh[f];
    const double* Xup = (Ss >= 0.0) ? qL : qR;
    for (int s = 0; s < P->nspec; s++) F[2 + dim + s] = Fh[0] * Xup[2 + dim + s];
}

/* MC limited slope (or the unlimited centred slope) from three values */
static double plm_slope(int limiter, double qm, double q0, double qp) {
    double dl = q0 - qm, dr = qp - q0, dc = 0.5 * (dl + dr);
    if (!limiter) return dc;
    if (dl * dr <= 0.0) return 0.0;
    double lim = fmin(2.0 * fabs(dl), 2.0 * fabs(dr));
    lim = fmin(lim, fabs(dc));
    return dc > 0.0 ? lim : -lim;
}

/* ------------------------------------------------------------------ */
/* Advective term A(U) (section 2: the divergence of the hydrodynamic */
/* fluxes), method of lines: cons->prim, PLM slopes per direction,    */
/* interface states, HLLC flux, flux difference.  Periodic box.        */
/* ------------------------------------------------------------------ */
void orc_advective(const orc_problem* P, const double* U, double* A) {
    int dim = P->dim, nv = orc_nvar(P), ns = P->nspec;
    long long N = nzones(P);
    double* q = (double*)malloc(sizeof(double) * nv * N);    /* zone-major primitives */
    double* F = (double*)malloc(sizeof(double) * nv * N);    /* face fluxes of one direction */
    for (long long z = 0; z < N; z++) cons_to_prim(P, U, N, z, q + z * nv);
    for (long long f = 0; f < (long long)nv * N; f++) A[f] = 0.0;

    for (int dir = 0; dir < dim; dir++) {
        int nd = P->n[dir];
        double dx = P->dx[dir];
        /* F[z*nv + f] = flux through the face between zone z and its +1 neighbour along dir */
#pragma omp parallel for schedule(static)
        for (long long z = 0; z < N; z++) {
            double qL[64], qR[64];
            int c[3];
            c[0] = (int)(z % P->n[0]);
            c[1] = (int)((z / P->n[0]) % P->n[1]);
            c[2] = (int)(z / ((long long)P->n[0] * P->n[1]));
            /* zones l-1, l, l+1, l+2 along dir around the face l+1/2 (l = this zone) */
            long long zz[4];
            for (int o = -1; o <= 2; o++) {
                int cc[3] = {c[0], c[1], c[2]};
                cc[dir] = ((c[dir] + o) % nd + nd) % nd;
                zz[o + 1] = IDX(P, cc[0], cc[1], cc[2]);
            }
            /* left state from zone l, right state from zone l+1 */
            for (int f = 0; f < nv; f++) {
                double sl = plm_slope(P->limiter, q[zz[0] * nv + f], q[zz[1] * nv + f], q[zz[2] * nv + f]);
                double sr = plm_slope(P->limiter, q[zz[1] * nv + f], q[zz[2] * nv + f], q[zz[3] * nv + f]);
                qL[f] = q[zz[1] * nv + f] + 0.5 * sl;
                qR[f] = q[zz[2] * nv + f] - 0.5 * sr;
            }
            /* interface mass fractions renormalised to sum to one */
            if (ns > 0) {
                double sL = 0.0, sR = 0.0;
                for (int s = 0; s < ns; s++) { sL += qL[2 + dim + s]; sR += qR[2 + dim + s]; }
                for (int s = 0; s < ns; s++) { qL[2 + dim + s] /= sL; qR[2 + dim + s] /= sR; }
            }
            orc_hllc(P, dir, qL, qR, F + z * nv);
        }
        /* A -= (F_{l+1/2} - F_{l-1/2}) / dx, directions accumulated in order x, y, z */
#pragma omp parallel for schedule(static)
        for (long long z = 0; z < N; z++) {
            int c[3];
            c[0] = (int)(z % P->n[0]);
            c[1] = (int)((z / P->n[0]) % P->n[1]);
            c[2] = (int)(z / ((long long)P->n[0] * P->n[1]));
            c[dir] = (c[dir] - 1 + nd) % nd;
            long long zm = IDX(P, c[0], c[1], c[2]);
            for (int f = 0; f < nv; f++) A[f * N + z] -= (F[z * nv + f] - F[zm * nv + f]) / dx;
        }
    }
    free(F);
    free(q);
}

/* ------------------------------------------------------------------ */
/* Fourth-order finite-volume operators (section 2: the fourth-order  */
/* method combines Simpson's rule with the spatial reconstruction of  */
/* McCorquodale & Colella).  Smooth-flow form (limiter = 0):         */
/*   point <-> average: f_c = <f> - L<f>/24,  <f> = f_c + L f_c/24,    */
/*     L = sum over the box's dimensions of the second difference;    */
/*   primitive averages <W> = W(U_c) + L W(<U>)/24;                   */
/*   face averages <W>_{i+1/2} = 7/12 (<W>_i + <W>_{i+1})              */
/*                             - 1/12 (<W>_{i-1} + <W>_{i+2});         */
/*   face-centre values W_f = <W>_{i+1/2} - L_t <W>_{i+1/2}/24, with   */
/*     L_t the second differences across the face (other dimensions); */
/*   face-average fluxes <F> = F(W_f) + L_t F(<W>_{i+1/2})/24;          */
/*   A = -sum_d (<F>_{i+1/2} - <F>_{i-1/2}) / dx_d.                    */
/* Both sides of a face see the same state, so F is the physical      */
/* Euler flux (species: mass flux times X).  Limited form (limiter =  */
/* 1): the face averages are limited per side (Colella & Sekora, see  */
/* cs_face / cs_zone below) and F is the HLLC flux between the two    */
/* sides, at the face centres and from the face averages alike.       */
/* ------------------------------------------------------------------ */
static long long shifted_zone(const orc_problem* P, long long z, int d, int o) {
    int c[3];
    c[0] = (int)(z % P->n[0]);
    c[1] = (int)((z / P->n[0]) % P->n[1]);
    c[2] = (int)(z / ((long long)P->n[0] * P->n[1]));
    c[d] = ((c[d] + o) % P->n[d] + P->n[d]) % P->n[d];
    return IDX(P, c[0], c[1], c[2]);
}

/* out = a + coef * sum_{d != skip} (b(z+e_d) - 2 b(z) + b(z-e_d)), field-major [nf][N] */
static void lap_combine(const orc_problem* P, int nf, const double* a, const double* b, double coef, int skip,
                        double* out) {
    long long N = nzones(P);
#pragma omp parallel for schedule(static)
    for (long long z = 0; z < N; z++) {
        long long zp[3], zm[3];
        for (int d = 0; d < P->dim; d++) {
            zp[d] = shifted_zone(P, z, d, 1);
            zm[d] = shifted_zone(P, z, d, -1);
        }
        for (int f = 0; f < nf; f++) {
            double l = 0.0;
            for (int d = 0; d < P->dim; d++) {
                if (d == skip) continue;
                l += b[f * N + zp[d]] - 2.0 * b[f * N + z] + b[f * N + zm[d]];
            }
            out[f * N + z] = a[f * N + z] + coef * l;
        }
    }
}

void orc_avg_to_point(const orc_problem* P, int nf, const double* avg, double* point) {
    lap_combine(P, nf, avg, avg, -1.0 / 24.0, -1, point);
}

void orc_point_to_avg(const orc_problem* P, int nf, const double* point, double* avg) {
    lap_combine(P, nf, point, point, 1.0 / 24.0, -1, avg);
}

/* primitives (rho, u, p, X) of every zone, field-major */
static void prim_fields(const orc_problem* P, const double* U, double* W) {
    int nv = orc_nvar(P);
    long long N = nzones(P);
#pragma omp parallel for schedule(static)
    for (long long z = 0; z < N; z++) {
        double q[64];
        cons_to_prim(P, U, N, z, q);
        for (int f = 0; f < nv; f++) W[f * N + z] = q[f];
    }
}

/* physical Euler flux along dir of the primitive state q */
static void euler_flux(const orc_problem* P, int dir, const double* q, double* F) {
    int dim = P->dim;
    double rho = q[0], un = q[1 + dir], p = q[1 + dim];
    double ke = 0.0;
    for (int d = 0; d < dim; d++) ke += 0.5 * rho * q[1 + d] * q[1 + d];
    double E = p / (P->gamma - 1.0) + ke;
    F[0] = rho * un;
    for (int d = 0; d < dim; d++) F[1 + d] = rho * un * q[1 + d] + (d == dir ? p : 0.0);
    F[1 + dim] = (E + p) * un;
    for (int s = 0; s < P->nspec; s++) F[2 + dim + s] = rho * un * q[2 + dim + s];
}

/* Limited form of the fourth-order face values (reading of the paper's
   fourth-order method for flows with steep fronts: the extremum-preserving PPM
   limiter of Colella & Sekora (2008) applied to the face values, then a
   Riemann solver between the two limited states of every face).  C = 1.25. */
#define CS_C 1.25

static int same_sign3(double a, double b, double c) {
    return (a > 0.0 && b > 0.0 && c > 0.0) || (a < 0.0 && b < 0.0 && c < 0.0);
}

/* face between zone i (a0) and i+1 (ap), neighbours am = a_{i-1}, app = a_{i+2}:
   a face value outside [a_i, a_{i+1}] is replaced by the mean of the two
   averages less a sixth of a limited second difference.  The face estimate
   d2f = 3 (a_i - 2 a_f + a_{i+1}) is h^2 f'' (exact on parabolas), and solving it
   for a_f gives a_f = (a_i + a_{i+1})/2 - d2f/6, so the replacement returns the
   face value unchanged wherever the limiter does not bind */
static double cs_face(double am, double a0, double ap, double app, double af) {
    if ((af - a0) * (ap - af) < 0.0) {
        double d2f = 3.0 * (a0 - 2.0 * af + ap);
        double d2l = am - 2.0 * a0 + ap, d2r = a0 - 2.0 * ap + app;
        double d2 = 0.0;
        if (same_sign3(d2f, d2l, d2r)) {
            double m = fmin(fmin(CS_C * fabs(d2l), CS_C * fabs(d2r)), fabs(d2f));
            d2 = d2f > 0.0 ? m : -m;
        }
        af = 0.5 * (a0 + ap) - d2 / 6.0;
    }
    return af;
}

/* zone i (average a0, neighbours amm..app) with face values *fm (i-1/2) and
   *fp (i+1/2): at an extremum (of the face values about the average, or of the
   averages at distance one or two) the deviations are scaled by a limited
   second derivative over the parabola's own; elsewhere the PPM overshoot limits
   apply.  The distance-two test catches an extremum that sits on a face of the
   zone: there the parabola meets the overshoot bound |dp| = 2 |dm| exactly, and
   the overshoot limit would clip smooth data by O(h^4) */
/* The extremum tests below compare the signs of two differences of averages
   on either side of the zone, e = a_left - a0 and e' = a0 - a_right.  Averages
   that mirror each other across a plane of symmetry of the data differ only by
   rounding, and a test would take its branch from the order of that rounding.
   A difference counts as zero (a tie) when it is at most 2^-20 of the other one
   or at most 2^-48 of the larger average it is formed from. */
#define CS_TIE_REL 20
#define CS_TIE_ABS 48
static double tie_diff(double d, double other, double a, double b) {
    if (fabs(d) <= ldexp(fabs(other), -CS_TIE_REL)) return 0.0;
    if (fabs(d) <= ldexp(fmax(fabs(a), fabs(b)), -CS_TIE_ABS)) return 0.0;
    return d;
}

/* e * e' <= 0 with ties counted as zero */
static int not_same_side(double al, double a0, double ar) {
    double e1 = al - a0, e2 = a0 - ar;
    double t1 = tie_diff(e1, e2, al, a0), t2 = tie_diff(e2, e1, a0, ar);
    return t1 * t2 <= 0.0;
}

static void cs_zone(double amm, double am, double a0, double ap, double app, double* fm, double* fp) {
    double dm = *fm - a0, dp = *fp - a0;
    if (dp * dm >= 0.0 || not_same_side(am, a0, ap) || not_same_side(amm, a0, app)) {
        double d2 = -2.0 * (6.0 * a0 - 3.0 * (*fm + *fp));
        double d2c = am - 2.0 * a0 + ap, d2l = amm - 2.0 * am + a0, d2r = a0 - 2.0 * ap + app;
        double lim = 0.0;
        if (same_sign3(d2, d2c, d2l) && same_sign3(d2, d2c, d2r)) {
            double m = fmin(fmin(fabs(d2), CS_C * fabs(d2c)), fmin(CS_C * fabs(d2l), CS_C * fabs(d2r)));
            lim = d2 > 0.0 ? m : -m;
        }
        if (d2 != 0.0) {
            *fm = a0 + dm * lim / d2;
            *fp = a0 + dp * lim / d2;
        } else {
            *fm = a0;
            *fp = a0;
        }
    } else {
        if (fabs(dp) >= 2.0 * fabs(dm)) *fp = a0 - 2.0 * dm;
        if (fabs(dm) >= 2.0 * fabs(dp)) *fm = a0 - 2.0 * dp;
    }
}

/* the limited left and right states of the face between z and its +1
   neighbour along dir (WL: zone z's upper face value, WR: zone z+1's lower
   one), from the averaged primitives Wa and the interpolated face values Wf */
static void limited_face_states(const orc_problem* P, int dir, const double* Wa, const double* Wf, double* WL,
                                double* WR) {
    int nv = orc_nvar(P);
    long long N = nzones(P);
    double* Wfl = (double*)malloc(sizeof(double) * nv * N);
#pragma omp parallel for schedule(static)
    for (long long z = 0; z < N; z++) {
        long long zm = shifted_zone(P, z, dir, -1), zp = shifted_zone(P, z, dir, 1), zpp = shifted_zone(P, z, dir, 2);
        for (int f = 0; f < nv; f++)
            Wfl[f * N + z] = cs_face(Wa[f * N + zm], Wa[f * N + z], Wa[f * N + zp], Wa[f * N + zpp], Wf[f * N + z]);
    }
#pragma omp parallel for schedule(static)
    for (long long z = 0; z < N; z++) {
        long long zmm = shifted_zone(P, z, dir, -2), zm = shifted_zone(P, z, dir, -1);
        long long zp = shifted_zone(P, z, dir, 1), zpp = shifted_zone(P, z, dir, 2);
        double qm[64], qp[64];
        for (int f = 0; f < nv; f++) {
            qm[f] = Wfl[f * N + zm];
            qp[f] = Wfl[f * N + z];
            cs_zone(Wa[f * N + zmm], Wa[f * N + zm], Wa[f * N + z], Wa[f * N + zp], Wa[f * N + zpp], &qm[f],
                    &qp[f]);
        }
        /* limited mass fractions renormalised to sum to one, as in the PLM states */
        if (P->nspec > 0) {
            double sm = 0.0, sp = 0.0;
            for (int s = 0; s < P->nspec; s++) { sm += qm[2 + P->dim + s]; sp += qp[2 + P->dim + s]; }
            for (int s = 0; s < P->nspec; s++) { qm[2 + P->dim + s] /= sm; qp[2 + P->dim + s] /= sp; }
        }
        for (int f = 0; f < nv; f++) {
            WL[f * N + z] = qp[f];   /* upper face of z */
            WR[f * N + zm] = qm[f];  /* lower face of z = upper face of z-1, seen from the right */
        }
    }
    free(Wfl);
}

/* limited_face_states on given averaged primitives Wa and face values Wf (a
   test hook for the limiter's properties) */
void orc_limited_faces(const orc_problem* P, int dir, const double* Wa, const double* Wf, double* WL, double* WR) {
    limited_face_states(P, dir, Wa, Wf, WL, WR);
}

void orc_advective4(const orc_problem* P, const double* U, double* A) {
    int dim = P->dim, nv = orc_nvar(P);
    long long N = nzones(P);
    size_t sz = sizeof(double) * nv * N;
    double *Uc = (double*)malloc(sz), *W2 = (double*)malloc(sz), *Wc = (double*)malloc(sz);
    double *Wa = (double*)malloc(sz), *Wf = (double*)malloc(sz), *Wfc = (double*)malloc(sz);
    double *Fc = (double*)malloc(sz), *F2 = (double*)malloc(sz), *Fa = (double*)malloc(sz);
    double *WL = NULL, *WR = NULL, *WLc = NULL, *WRc = NULL;
    if (P->limiter) {
        WL = (double*)malloc(sz); WR = (double*)malloc(sz);
        WLc = (double*)malloc(sz); WRc = (double*)malloc(sz);
    }
    orc_avg_to_point(P, nv, U, Uc);
    prim_fields(P, U, W2);
    prim_fields(P, Uc, Wc);
    lap_combine(P, nv, Wc, W2, 1.0 / 24.0, -1, Wa);
    for (long long f = 0; f < (long long)nv * N; f++) A[f] = 0.0;
    for (int dir = 0; dir < dim; dir++) {
        /* face between zone z and its +1 neighbour along dir, indexed by z */
#pragma omp parallel for schedule(static)
        for (long long z = 0; z < N; z++) {
            long long zm = shifted_zone(P, z, dir, -1), zp = shifted_zone(P, z, dir, 1),
                      zpp = shifted_zone(P, z, dir, 2);
            for (int f = 0; f < nv; f++)
                Wf[f * N + z] = 7.0 / 12.0 * (Wa[f * N + z] + Wa[f * N + zp]) -
                                1.0 / 12.0 * (Wa[f * N + zm] + Wa[f * N + zpp]);
        }
        if (P->limiter) {
            /* limited: the two states of every face, then HLLC between them at the
               face centres (transverse maps of each side) and from the averages */
            limited_face_states(P, dir, Wa, Wf, WL, WR);
            lap_combine(P, nv, WL, WL, -1.0 / 24.0, dir, WLc);
            lap_combine(P, nv, WR, WR, -1.0 / 24.0, dir, WRc);
#pragma omp parallel for schedule(static)
            for (long long z = 0; z < N; z++) {
                double qL[64], qR[64], F[64];
                for (int f = 0; f < nv; f++) { qL[f] = WLc[f * N + z]; qR[f] = WRc[f * N + z]; }
                orc_hllc(P, dir, qL, qR, F);
                for (int f = 0; f < nv; f++) Fc[f * N + z] = F[f];
                for (int f = 0; f < nv; f++) { qL[f] = WL[f * N + z]; qR[f] = WR[f * N + z]; }
                orc_hllc(P, dir, qL, qR, F);
                for (int f = 0; f < nv; f++) F2[f * N + z] = F[f];
            }
        } else {
            lap_combine(P, nv, Wf, Wf, -1.0 / 24.0, dir, Wfc);
#pragma omp parallel for schedule(static)
            for (long long z = 0; z < N; z++) {
                double q[64], F[64];
                for (int f = 0; f < nv; f++) q[f] = Wfc[f * N + z];
                euler_flux(P, dir, q, F);
                for (int f = 0; f < nv; f++) Fc[f * N + z] = F[f];
                for (int f = 0; f < nv; f++) q[f] = Wf[f * N + z];
                euler_flux(P, dir, q, F);
                for (int f = 0; f < nv; f++) F2[f * N + z] = F[f];
            }
        }
        lap_combine(P, nv, Fc, F2, 1.0 / 24.0, dir, Fa);
        double dx = P->dx[dir];
#pragma omp parallel for schedule(static)
        for (long long z = 0; z < N; z++) {
            long long zm = shifted_zone(P, z, dir, -1);
            for (int f = 0; f < nv; f++) A[f * N + z] -= (Fa[f * N + z] - Fa[f * N + zm]) / dx;
        }
    }
    free(Uc); free(W2); free(Wc); free(Wa); free(Wf); free(Wfc); free(Fc); free(F2); free(Fa);
    free(WL); free(WR); free(WLc); free(WRc);
}

void orc_advective_term(const orc_problem* P, const double* U, double* A) {
    if (P->space_order == 4) orc_advective4(P, U, A);
    else orc_advective(P, U, A);
}

/* ------------------------------------------------------------------ */
/* Reaction network: rates, sources R(w) and the analytic dR/dw.      */
/* w = [rho E, rho X_0 .. rho X_{nspec-1}] at one zone; rho and the   */
/* momenta are parameters (R has no mass or momentum component).      */
/*   Y_i = X_i / mass_i,  T from the gamma-law EOS,                    */
/*   r_j = a_j rho^(o_j-1) f_j(T) prod Y^cnt,                          */
/*   R(rho X_i) = rho mass_i sum_j s_ij r_j,  R(rho E) = rho sum Q_j r_j */
/* ------------------------------------------------------------------ */
static double ipow(double x, int c) {
    double r = 1.0;
    for (int i = 0; i < c; i++) r *= x;
    return r;
}

void orc_rates(const orc_problem* P, double rho, const double* mom, const double* w,
               double* R, double* dRdw) {
    int ns = P->nspec, n = ns + 1;
    double T = orc_temperature(P, rho, mom, w[0]);
    double dTdE = (P->gamma - 1.0) / rho;
    double Y[ORC_MAX_SPEC];
    for (int i = 0; i < ns; i++) Y[i] = w[1 + i] / (rho * P->mass[i]);
    for (int r = 0; r < n; r++) R[r] = 0.0;
    if (dRdw)
        for (int r = 0; r < n * n; r++) dRdw[r] = 0.0;

    for (int j = 0; j < P->nreac; j++) {
        int order = 0;
        for (int s = 0; s < 2; s++)
            if (P->reac[j][s] >= 0) order += P->cnt[j][s];
        double rho_pow = ipow(rho, order - 1);
        double f, dfdT;
        if (P->rate_law == ORC_RATE_POWER) {
            f = pow(T, P->nu[j]);
            dfdT = P->nu[j] * f / T;
        } else {
            f = exp(-P->nu[j] / T);
            dfdT = f * P->nu[j] / (T * T);
        }
        double prodY = 1.0;
        for (int s = 0; s < 2; s++)
            if (P->reac[j][s] >= 0) prodY *= ipow(Y[P->reac[j][s]], P->cnt[j][s]);
        double rate = P->a[j] * rho_pow * f * prodY;

        /* stoichiometric change of every species in reaction j */
        double sto[ORC_MAX_SPEC];
        for (int i = 0; i < ns; i++) sto[i] = 0.0;
        for (int s = 0; s < 2; s++)
            if (P->reac[j][s] >= 0) sto[P->reac[j][s]] -= P->cnt[j][s];
        sto[P->prod[j]] += 1.0;

        R[0] += rho * P->Q[j] * rate;
        for (int i = 0; i < ns; i++) R[1 + i] += rho * P->mass[i] * sto[i] * rate;

        if (dRdw) {
            /* d rate / d w_c */
            double drdw[ORC_MAX_SPEC + 1];
            for (int c = 0; c < n; c++) drdw[c] = 0.0;
            drdw[0] = P->a[j] * rho_pow * dfdT * prodY * dTdE;
            for (int s = 0; s < 2; s++) {
                int k = P->reac[j][s];
                if (k < 0) continue;
                double dprod = P->cnt[j][s] * ipow(Y[k], P->cnt[j][s] - 1);
                int o = 1 - s;
                if (P->reac[j][o] >= 0) dprod *= ipow(Y[P->reac[j][o]], P->cnt[j][o]);
                drdw[1 + k] += P->a[j] * rho_pow * f * dprod / (rho * P->mass[k]);
            }
            for (int c = 0; c < n; c++) {
                dRdw[0 * n + c] += rho * P->Q[j] * drdw[c];
                for (int i = 0; i < ns; i++) dRdw[(1 + i) * n + c] += rho * P->mass[i] * sto[i] * drdw[c];
            }
        }
    }
}

void orc_reaction_source(const orc_problem* P, const double* U, double* R) {
    int dim = P->dim, n = P->nspec + 1;
    long long N = nzones(P);
#pragma omp parallel for schedule(static)
    for (long long z = 0; z < N; z++) {
        double mom[3], w[ORC_MAX_SPEC + 1], Rz[ORC_MAX_SPEC + 1];
        double rho = U[z];
        for (int d = 0; d < dim; d++) mom[d] = U[(1 + d) * N + z];
        for (int r = 0; r < n; r++) w[r] = U[(1 + dim + r) * N + z];
        orc_rates(P, rho, mom, w, Rz, NULL);
        for (int r = 0; r < n; r++) R[r * N + z] = Rz[r];
    }
}

/* ------------------------------------------------------------------ */
/* Dense LU with partial pivoting (largest |entry|, ties to the lowest */
/* row index) and the triangular solves.  Returns -1 on a zero pivot. */
/* ------------------------------------------------------------------ */
static int lu_solve(int n, double* J, double* b) {
    for (int k = 0; k < n; k++) {
        int piv = k;
        double best = fabs(J[k * n + k]);
        for (int i = k + 1; i < n; i++)
            if (fabs(J[i * n + k]) > best) { best = fabs(J[i * n + k]); piv = i; }
        if (best == 0.0) return -1;
        if (piv != k) {
            for (int c = 0; c < n; c++) {
                double t = J[k * n + c]; J[k * n + c] = J[piv * n + c]; J[piv * n + c] = t;
            }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int i = k + 1; i < n; i++) {
            double l = J[i * n + k] / J[k * n + k];
            J[i * n + k] = l;
            for (int c = k + 1; c < n; c++) J[i * n + c] -= l * J[k * n + c];
            b[i] -= l * b[k];
        }
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = b[i];
        for (int c = i + 1; c < n; c++) s -= J[i * n + c] * b[c];
        b[i] = s / J[i * n + i];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Implicit reaction update (section 2: the reactive part of the node */
/* update is implicit in the new state).  Solve                         */
/*   G(w) = w - dt_m R(w) - rhs_w = 0,   J_G = I - dt_m dR/dw          */
/* by Newton iteration, globalised by pseudo-transient continuation:   */
/* an iteration solves (c I - dt_m dR/dw) delta = G(w) with c = 1 for a */
/* Newton step and c = 1 + 1/h for a pseudo-time step of size h of      */
/* dw/dtau = -G(w) (the burning ODE relaxed towards rhs), then sets     */
/* w <- w - delta.                                                     */
/*   - start in Newton mode;                                           */
/*   - a trial is admissible when T > 0 (finite) and, if every rhs mass */
/*     fraction is >= -0.01, every mass fraction stays above            */
/*     min(0, X_i of rhs, X_i of the start) - 0.01 (a wide floor: it    */
/*     stops excursions into grossly negative compositions, not the     */
/*     small negative values a root can have; an rhs already pushed     */
/*     further negative by the correction terms gets no floor);         */
/*   - a start without a positive temperature is replaced by rhs;       */
/*   - a Newton trial that is not admissible or raises the scaled       */
/*     residual norm switches to pseudo mode with h = 1 (w unchanged);  */
/*   - in pseudo mode an admissible trial is taken and h grows x3, a    */
/*     trial that is not admissible is dropped and h shrinks /4; once   */
/*     h >= 1e3 the solve returns to Newton mode;                       */
/*   - converged when a Newton step was taken with                      */
/*     max(|d(rhoE)|/|rhoE|, max_i |d(rho X_i)|/rho) <= rtol.           */
/* Every pass of the loop (one linear solve) counts as one iteration.  */
/* ------------------------------------------------------------------ */
#define PTC_H0 1.0
#define PTC_GROW 3.0
#define PTC_SHRINK 4.0
#define PTC_HNEWTON 1e3
#define PTC_HMIN 1e-12
#define NEWTON_XMARGIN 1e-2

static double scaled_norm2(int n, const double* G, double sE, double rho) {
    double s = (G[0] / sE) * (G[0] / sE);
    for (int i = 1; i < n; i++) s += (G[i] / rho) * (G[i] / rho);
    return s;
}

int orc_newton_zone(const orc_problem* P, double rho, const double* mom, const double* rhs_w,
                    double dt_m, double* w, int* iters) {
    int ns = P->nspec, n = ns + 1;
    double R[ORC_MAX_SPEC + 1], dR[(ORC_MAX_SPEC + 1) * (ORC_MAX_SPEC + 1)];
    double Rt[ORC_MAX_SPEC + 1], dRt[(ORC_MAX_SPEC + 1) * (ORC_MAX_SPEC + 1)];
    double M[(ORC_MAX_SPEC + 1) * (ORC_MAX_SPEC + 1)], G[ORC_MAX_SPEC + 1], Gt[ORC_MAX_SPEC + 1];
    double d[ORC_MAX_SPEC + 1], trial[ORC_MAX_SPEC + 1], lower[ORC_MAX_SPEC];
    double sE = fabs(rhs_w[0]);
    /* a guess without a positive temperature is replaced by rhs */
    double Tg = orc_temperature(P, rho, mom, w[0]);
    if (!(Tg > 0.0 && Tg < INFINITY))
        for (int r = 0; r < n; r++) w[r] = rhs_w[r];
    /* the floor applies when the rhs is physical (every X_i >= -0.01); an rhs
       that the correction terms pushed further negative has no floor */
    int physical = 1;
    for (int i = 0; i < ns; i++)
        if (!(rhs_w[1 + i] / rho >= -NEWTON_XMARGIN)) physical = 0;
    for (int i = 0; i < ns; i++) {
        double x = rhs_w[1 + i] / rho, xg = w[1 + i] / rho;
        double lo = x < 0.0 ? x : 0.0;
        if (xg < lo) lo = xg;
        lower[i] = physical ? lo - NEWTON_XMARGIN : -INFINITY;
    }
    double T0 = orc_temperature(P, rho, mom, w[0]);
    if (!(T0 > 0.0 && T0 < INFINITY)) { *iters = 0; return ORC_NEWTON_NONPHYSICAL; }
    orc_rates(P, rho, mom, w, R, dR);
    for (int r = 0; r < n; r++) G[r] = w[r] - dt_m * R[r] - rhs_w[r];
    double phi = scaled_norm2(n, G, sE, rho);
    int newton = 1;
    double h = PTC_H0;
    int status = ORC_NEWTON_MAXIT;
    int it;
    for (it = 1; it <= P->newton_maxit; it++) {
        double c = newton ? 1.0 : 1.0 + 1.0 / h;
        for (int r = 0; r < n; r++) {
            for (int col = 0; col < n; col++) M[r * n + col] = (r == col ? c : 0.0) - dt_m * dR[r * n + col];
            d[r] = G[r];
        }
        if (lu_solve(n, M, d) != 0) { status = ORC_NEWTON_SINGULAR; break; }
        for (int r = 0; r < n; r++) trial[r] = w[r] - d[r];
        double T = orc_temperature(P, rho, mom, trial[0]);
        int ok = T > 0.0 && T < INFINITY;
        for (int i = 0; i < ns && ok; i++)
            if (!(trial[1 + i] / rho >= lower[i])) ok = 0;
        double phit = 0.0;
        if (ok) {
            orc_rates(P, rho, mom, trial, Rt, dRt);
            for (int r = 0; r < n; r++) Gt[r] = trial[r] - dt_m * Rt[r] - rhs_w[r];
            phit = scaled_norm2(n, Gt, sE, rho);
            if (!(phit < INFINITY)) ok = 0;
        }
        /* the Newton step meets the stop test: converged (a residual that grew
           by round-off at the root does not count against it) */
        int small = 0;
        if (newton && ok) {
            double err = fabs(d[0]) / fabs(trial[0]);
            for (int i = 0; i < ns; i++) {
                double e = fabs(d[1 + i]) / rho;
                if (e > err) err = e;
            }
            small = err <= P->newton_rtol;
        }
        if (newton && !small && (!ok || phit > phi)) {
            newton = 0;
            h = PTC_H0;
            continue;
        }
        if (!ok) {
            h /= PTC_SHRINK;
            if (h < PTC_HMIN) { status = ORC_NEWTON_NONPHYSICAL; break; }
            continue;
        }
        for (int r = 0; r < n; r++) {
            w[r] = trial[r];
            R[r] = Rt[r];
            G[r] = Gt[r];
        }
        for (int r = 0; r < n * n; r++) dR[r] = dRt[r];
        phi = phit;
        if (newton) {
            double err = fabs(d[0]) / fabs(w[0]);
            for (int i = 0; i < ns; i++) {
                double e = fabs(d[1 + i]) / rho;
                if (e > err) err = e;
            }
            if (err <= P->newton_rtol) { status = ORC_NEWTON_OK; break; }
        } else {
            h *= PTC_GROW;
            if (h >= PTC_HNEWTON) newton = 1;
        }
    }
    if (it > P->newton_maxit) it = P->newton_maxit;
    *iters = it;
    return status;
}

void orc_react_newton(const orc_problem* P, const double* rhs, double dt_m, double* U_inout,
                      double* R_out, int* zone_status, int* zone_iters, orc_stats* st) {
    int dim = P->dim, n = P->nspec + 1;
    long long N = nzones(P);
    long long tot = 0, fail = 0;
    long long hist[64] = {0};
#pragma omp parallel
    {
        long long ltot = 0, lfail = 0;
        long long lhist[64] = {0};
#pragma omp for schedule(dynamic, 64)
        for (long long z = 0; z < N; z++) {
            double mom[3], w[ORC_MAX_SPEC + 1], rw[ORC_MAX_SPEC + 1], Rz[ORC_MAX_SPEC + 1];
            double rho = rhs[z];
            for (int d = 0; d < dim; d++) mom[d] = rhs[(1 + d) * N + z];
            /* the guess keeps the specific values (X_i, E) of the previous iterate
               and takes the density of the right-hand side */
            double scale = rho / U_inout[z];
            for (int r = 0; r < n; r++) {
                rw[r] = rhs[(1 + dim + r) * N + z];
                w[r] = U_inout[(1 + dim + r) * N + z] * scale;
            }
            int iters = 0;
            int s = orc_newton_zone(P, rho, mom, rw, dt_m, w, &iters);
            orc_rates(P, rho, mom, w, Rz, NULL);
            U_inout[z] = rho;
            for (int d = 0; d < dim; d++) U_inout[(1 + d) * N + z] = mom[d];
            for (int r = 0; r < n; r++) {
                U_inout[(1 + dim + r) * N + z] = w[r];
                R_out[r * N + z] = Rz[r];
            }
            if (zone_status) zone_status[z] = s;
            if (zone_iters) zone_iters[z] = iters;
            ltot += iters;
            if (s != ORC_NEWTON_OK) lfail++;
            lhist[iters < 63 ? iters : 63]++;
        }
#pragma omp critical
        {
            tot += ltot;
            fail += lfail;
            for (int i = 0; i < 64; i++) hist[i] += lhist[i];
        }
    }
    if (st) {
        st->newton_iters_total += tot;
        st->newton_solves += N;
        st->n_fail += fail;
        for (int i = 0; i < 64; i++) st->hist[i] += hist[i];
    }
}

/* ------------------------------------------------------------------ */
/* Node-to-node integral I_m = sum_l q_{m,l} dt (A_l + R_l)            */
/* ------------------------------------------------------------------ */
/* Fourth order: the average of the source is R at the zone-centre state
   plus the Laplacian correction, <R> = R(U_c) + L R(U_c)/24, U_c = <U> - L<U>/24. */
void orc_reaction_source4(const orc_problem* P, const double* U, double* R) {
    int nv = orc_nvar(P), n = P->nspec + 1;
    long long N = nzones(P);
    double* Uc = (double*)malloc(sizeof(double) * nv * N);
    double* Rc = (double*)malloc(sizeof(double) * n * N);
    orc_avg_to_point(P, nv, U, Uc);
    orc_reaction_source(P, Uc, Rc);
    orc_point_to_avg(P, n, Rc, R);
    free(Uc);
    free(Rc);
}

/* Fourth-order implicit update of the average equation
   <U> - dt_m <R(U)> = <rhs>.  The map f -> f - L f/24 (linear, averages to
   zone centres to fourth order) turns it into U_c - dt_m R(U_c) = rhs_c, solved
   zone by zone as in the second-order update (guess: the centre values of the
   guess); its source is mapped back, <R> = R_c + L R_c/24, and the averages
   are <U> = <rhs> + dt_m <R> (mass and momenta: <rhs>).  Mapping the centre
   state itself back instead would add (I + L/24)(I - L/24) - I = -L^2/576, an
   O(h^4) change per solve even where nothing burns. */
void orc_react_newton4(const orc_problem* P, const double* rhs, double dt_m, double* U_inout, double* R_out,
                       orc_stats* st) {
    int nv = orc_nvar(P), n = P->nspec + 1, dim = P->dim;
    long long N = nzones(P);
    double* rc = (double*)malloc(sizeof(double) * nv * N);
    double* gc = (double*)malloc(sizeof(double) * nv * N);
    double* Rc = (double*)malloc(sizeof(double) * n * N);
    orc_avg_to_point(P, nv, rhs, rc);
    orc_avg_to_point(P, nv, U_inout, gc);
    orc_react_newton(P, rc, dt_m, gc, Rc, NULL, NULL, st);
    orc_point_to_avg(P, n, Rc, R_out);
    for (int f = 0; f < nv; f++)
        for (long long z = 0; z < N; z++) {
            double v = rhs[f * N + z];
            if (f >= 1 + dim) v += dt_m * R_out[(f - 1 - dim) * N + z];
            U_inout[f * N + z] = v;
        }
    free(rc);
    free(gc);
    free(Rc);
}

void orc_node_integral(const orc_problem* P, const double* const* A_nodes,
                       const double* const* R_nodes, double dt, int m, double* I) {
    int M = P->n_nodes, dim = P->dim, nv = orc_nvar(P);
    long long N = nzones(P);
    double q[64];
    orc_quad_weights(P->node_type, M, q);
    for (int f = 0; f < nv; f++)
        for (long long z = 0; z < N; z++) {
            double s = 0.0;
            for (int l = 0; l < M; l++) {
                double src = A_nodes[l][f * N + z];
                if (f >= 1 + dim) src += R_nodes[l][(f - 1 - dim) * N + z];
                s += q[m * M + l] * dt * src;
            }
            I[f * N + z] = s;
        }
}

/* ------------------------------------------------------------------ */
/* One SDC time step (section 2, Eq. sdc:general).                     */
/*   iterate 0: every node holds U^n, A and R evaluated there;         */
/*   iteration k -> k+1: node 0 stays U^n; for m = 0..M-2               */
/*     A^{m,(k+1)} = A(U^{m,(k+1)})                                    */
/*     rhs = U^{m,(k+1)} + dt_m (A^{m,(k+1)} - A^{m,(k)})               */
/*           - dt_m R^{m+1,(k)} + I_m[(k)]                             */
/*     U^{m+1,(k+1)} - dt_m R(U^{m+1,(k+1)}) = rhs  (Newton, guess      */
/*     U^{m+1,(k)}), R^{m+1,(k+1)} = R(U^{m+1,(k+1)});                   */
/*   A at the last node is evaluated for the next iteration's integral. */
/*   U^{n+1} = U^{M-1,(K)}.                                             */
/* ------------------------------------------------------------------ */
/* the operators of one sub-problem: A = 0 when only reactions run, R = 0
   (and the implicit update w = rhs) when only advection runs */
static void step_advective(const orc_problem* P, const double* U, double* A) {
    if (P->split_op == ORC_OP_REACT) {
        memset(A, 0, sizeof(double) * orc_nvar(P) * nzones(P));
        return;
    }
    orc_advective_term(P, U, A);
}

static void step_source(const orc_problem* P, const double* U, double* R) {
    if (P->split_op == ORC_OP_ADVECT) {
        memset(R, 0, sizeof(double) * (P->nspec + 1) * nzones(P));
        return;
    }
    if (P->space_order == 4) orc_reaction_source4(P, U, R);
    else orc_reaction_source(P, U, R);
}

/* The Newton guess of the node update (the paper does not say how the
   implicit equation is started).  The explicit predictor: the update of
   Eq. sdc:general with the unknown R^{m+1,(k+1)} replaced by the previous
   iterate's R^{m+1,(k)}, that is rhs + dt_m R^{m+1,(k)} in the reactive fields
   (R(U^n) in the first iteration), with rho and rho u of the rhs.  Where that
   state has no positive temperature or a mass fraction below -0.01, the guess
   stays the previous iterate U^{m+1,(k)} (U^n in the first iteration), as G
   holds it on entry. */
static void newton_guess(const orc_problem* P, const double* rhs, const double* Rk, double dtm, double* G) {
    int dim = P->dim, nv = orc_nvar(P), n = P->nspec + 1;
    long long N = nzones(P);
#pragma omp parallel for schedule(static)
    for (long long z = 0; z < N; z++) {
        double g[64];
        for (int f = 0; f < nv; f++) g[f] = rhs[f * N + z];
        for (int r = 0; r < n; r++) g[1 + dim + r] += dtm * Rk[r * N + z];
        int ok = orc_temperature(P, g[0], g + 1, g[1 + dim]) > 0.0;
        for (int i = 0; i < P->nspec; i++)
            if (g[2 + dim + i] < -1e-2 * g[0]) ok = 0;
        if (ok)
            for (int f = 0; f < nv; f++) G[f * N + z] = g[f];
    }
}

static void step_implicit(const orc_problem* P, const double* rhs, double dtm, double* U, double* R,
                          orc_stats* st) {
    if (P->split_op == ORC_OP_ADVECT) {
        memcpy(U, rhs, sizeof(double) * orc_nvar(P) * nzones(P));
        memset(R, 0, sizeof(double) * (P->nspec + 1) * nzones(P));
        return;
    }
    if (P->space_order == 4) orc_react_newton4(P, rhs, dtm, U, R, st);
    else orc_react_newton(P, rhs, dtm, U, R, NULL, NULL, st);
}

int orc_sdc_step_nodes(const orc_problem* P, double* U, double dt, orc_stats* st, double* nodes_out) {
    int M = P->n_nodes, K = P->n_iters, dim = P->dim, nv = orc_nvar(P), n = P->nspec + 1;
    long long N = nzones(P);
    double tau[8];
    if (orc_nodes(P->node_type, M, tau) != 0) return -1;
    size_t sz_u = sizeof(double) * nv * N, sz_r = sizeof(double) * n * N;
    double *Un[8], *Aold[8], *Anew[8], *Rold[8], *Rnew[8];
    for (int m = 0; m < M; m++) {
        Un[m] = (double*)malloc(sz_u);
        Aold[m] = (double*)malloc(sz_u);
        Anew[m] = (double*)malloc(sz_u);
        Rold[m] = (double*)malloc(sz_r);
        Rnew[m] = (double*)malloc(sz_r);
    }
    double* rhs = (double*)malloc(sz_u);
    double* I = (double*)malloc(sz_u);

    /* iterate 0 */
    for (int m = 0; m < M; m++) memcpy(Un[m], U, sz_u);
    step_advective(P, U, Aold[0]);
    step_source(P, U, Rold[0]);
    for (int m = 1; m < M; m++) {
        memcpy(Aold[m], Aold[0], sz_u);
        memcpy(Rold[m], Rold[0], sz_r);
    }
    int rc = 0;
    for (int k = 0; k < K; k++) {
        /* node 0 is U^n at every iteration, so its A and R do not change */
        memcpy(Anew[0], Aold[0], sz_u);
        memcpy(Rnew[0], Rold[0], sz_r);
        for (int m = 0; m < M - 1; m++) {
            double dtm = dt * (tau[m + 1] - tau[m]);
            if (m > 0) step_advective(P, Un[m], Anew[m]);
            orc_node_integral(P, (const double* const*)Aold, (const double* const*)Rold, dt, m, I);
            for (int f = 0; f < nv; f++)
                for (long long z = 0; z < N; z++) {
                    double v = Un[m][f * N + z] + dtm * (Anew[m][f * N + z] - Aold[m][f * N + z]);
                    if (f >= 1 + dim) v -= dtm * Rold[m + 1][(f - 1 - dim) * N + z];
                    rhs[f * N + z] = v + I[f * N + z];
                }
            /* Un[m+1] holds U^{m+1,(k)}, takes the guess and receives U^{m+1,(k+1)} */
            if (P->split_op != ORC_OP_ADVECT) newton_guess(P, rhs, Rold[m + 1], dtm, Un[m + 1]);
            step_implicit(P, rhs, dtm, Un[m + 1], Rnew[m + 1], st);
        }
        if (k < K - 1) step_advective(P, Un[M - 1], Anew[M - 1]);
        for (int m = 0; m < M; m++) {
            double* t = Aold[m]; Aold[m] = Anew[m]; Anew[m] = t;
            t = Rold[m]; Rold[m] = Rnew[m]; Rnew[m] = t;
        }
    }
    memcpy(U, Un[M - 1], sz_u);
    if (nodes_out)
        for (int m = 0; m < M; m++) memcpy(nodes_out + (size_t)m * nv * N, Un[m], sz_u);
    for (int m = 0; m < M; m++) {
        free(Un[m]); free(Aold[m]); free(Anew[m]); free(Rold[m]); free(Rnew[m]);
    }
    free(rhs);
    free(I);
    return rc;
}

int orc_sdc_step(const orc_problem* P, double* U, double dt, orc_stats* st) {
    return orc_sdc_step_nodes(P, U, dt, st, NULL);
}

int orc_strang_step(const orc_problem* P, double* U, double dt, orc_stats* st) {
    orc_problem Pr = *P, Pa = *P;
    Pr.split_op = ORC_OP_REACT;
    Pa.split_op = ORC_OP_ADVECT;
    if (orc_sdc_step(&Pr, U, 0.5 * dt, st) != 0) return -1;
    if (orc_sdc_step(&Pa, U, dt, st) != 0) return -1;
    return orc_sdc_step(&Pr, U, 0.5 * dt, st);
}

double orc_cfl_dt(const orc_problem* P, const double* U, double cfl) {
    int dim = P->dim, nv = orc_nvar(P);
    long long N = nzones(P);
    double smax = 0.0;
    double q[64];
    for (long long z = 0; z < N; z++) {
        cons_to_prim(P, U, N, z, q);
        double c = sqrt(P->gamma * q[1 + dim] / q[0]);
        double s = 0.0;
        for (int d = 0; d < dim; d++) s += (fabs(q[1 + d]) + c) / P->dx[d];
        if (s > smax) smax = s;
    }
    (void)nv;
    return cfl / smax;
}
