// sdc_dev.cuh -- device-side building blocks of the SDC hot path on sm_103a:
// network parameters, gamma-law EOS, rate constants, reactive sources and
// their Jacobian, and the dense pivoted LU of the implicit reaction update.
//
// Paper: arXiv:1910.12578, section 2 (Eq. 1, Eq. sdc:general).  The network,
// EOS and Newton globalisation are the readings stated in sdc.h:
// r_j = a_j rho^(o_j-1) f_j(T) prod Y^cnt, p = rho T, e = T/(gamma-1).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sdc_fastmath.cuh"
#include "sdc_pow.cuh"

#define SDCD_MAXS 16
#define SDCD_MAXR 16

namespace sdcd {

// temporal nodes of a step, at most (Radau: node 0 and three Radau IIA points)
constexpr int MAXM = 4;

enum { TOPO_GENERIC = 0, TOPO_CHAIN = 1 };
enum { LAW_POWER = 0, LAW_ARRHENIUS = 1 };
enum { ZONE_OK = 0, ZONE_MAXIT = 1, ZONE_NONPHYSICAL = 2, ZONE_SINGULAR = 3 };

// Network and gas constants, passed by value to every kernel.
struct NetParams {
    int nspec, nreac, law, topo;
    double gm1;                          // gamma - 1
    double gm1_inv;                      // 1 / (gamma - 1)
    double gamma;
    double mass[SDCD_MAXS];
    double inv_mass[SDCD_MAXS];
    double a[SDCD_MAXR], nu[SDCD_MAXR], Q[SDCD_MAXR];
    int r0[SDCD_MAXR], c0[SDCD_MAXR], r1[SDCD_MAXR], c1[SDCD_MAXR], prod[SDCD_MAXR];
    int order[SDCD_MAXR];                // sum of reactant multiplicities
    // alpha chain: a_j / prod_reactants mass (with multiplicity), so that
    // rho r_j = amp_j f_j(T) prod_reactants (rho X)^count
    double amp[SDCD_MAXR];
    // alpha chain with the power law and every nu_j <= 45: the rate factors of a
    // state within 2^-32 of a known one in T may be carried to first order
    int rate_taylor;
    // alpha chain: reaction j's share of the Newton matrix, per row (E, X_0, the
    // consumed X_j, the product X_{j+1}) and column (E, X_0, X_j); see build_chain
    double kc[SDCD_MAXR][12];
    // alpha chain: reaction j's coefficients in the sources, mass_i s_ij for
    // i = X_0, the consumed X_j (none for j = 0) and the product X_{j+1}
    double rs[SDCD_MAXR][3];
    float kcf[SDCD_MAXR][12];
    float kcl[SDCD_MAXR][12];  // kc - kcf: the float pair (kcf, kcl) of the FP32-pair matrix
};

// Coefficients of build_chain from the masses and energies of the alpha chain
// (j = 0: 3 A_0 -> A_1; j >= 1: A_j + A_0 -> A_{j+1}), and the prefactors amp.
// In terms of the unknowns w (rho E, rho X_i) the rates are
// r_j = kappa_j prod_reactants w^count with kappa_j = (amp_j / rho) f_j(T):
// the species masses and the density of Y_i = w_i / (rho mass_i) are folded
// into kappa_j.  Row i of dR/dw takes rho sigma_ij dr_j/dw (sigma_ij = Q_j in
// the energy row, mass_i s_ij in species row i), so entry (i, c) of
// M = c I - dt_m dR/dw gains -sigma_ij times dt_m rho kappa_j dP_j/dw_c
// (P_j = prod w), and entry (i, E) gains -sigma_ij times
// dt_m (gamma-1) f r_j nu_j (dr_j/d(rho E) = nu_j r_j f (gamma-1)/rho with
// f = 1/T for the power law, 1/T^2 for the Arrhenius law).  For j = 0 the
// factor 3 of dP_0/dw_0 = 3 w_0^2 is folded into the X_0 column's
// coefficients, and nu_j into the E column's.
inline void set_chain_coefs(NetParams& P) {
    for (int j = 0; j < SDCD_MAXR; j++) {
        P.amp[j] = 0.0;
        for (int e = 0; e < 12; e++) P.kc[j][e] = 0.0;
        for (int e = 0; e < 12; e++) P.kcf[j][e] = P.kcl[j][e] = 0.0f;
        P.rs[j][0] = P.rs[j][1] = P.rs[j][2] = 0.0;
    }
    P.rate_taylor = 0;
    if (P.topo != TOPO_CHAIN) return;
    P.rate_taylor = P.law == LAW_POWER;
    for (int j = 0; j < P.nreac; j++)
        if (!(P.nu[j] >= 0.0 && P.nu[j] <= 45.0)) P.rate_taylor = 0;
    const double* m = P.mass;
    for (int j = 0; j < P.nreac; j++) {
        P.amp[j] = j == 0 ? P.a[0] / (m[0] * m[0] * m[0]) : P.a[j] / (m[j] * m[0]);
        P.rs[j][0] = (j == 0 ? -3.0 : -1.0) * m[0];
        P.rs[j][1] = j == 0 ? 0.0 : -m[j];
        P.rs[j][2] = m[j + 1];
        double* c = P.kc[j];
        const double f0 = j == 0 ? 3.0 : 1.0;        // dP/dw_0 = f0 * (w_0^2 or w_j)
        const double s0 = j == 0 ? -3.0 : -1.0;      // stoichiometry of A_0
        // row E
        c[0] = P.Q[j];
        c[1] = f0 * P.Q[j];
        c[2] = j == 0 ? 0.0 : P.Q[j];
        // row X_0
        c[3] = s0 * m[0];
        c[4] = f0 * s0 * m[0];
        c[5] = j == 0 ? 0.0 : s0 * m[0];
        // row X_j (consumed; none for j = 0)
        c[6] = j == 0 ? 0.0 : -m[j];
        c[7] = j == 0 ? 0.0 : -m[j];
        c[8] = j == 0 ? 0.0 : -m[j];
        // row X_{j+1} (made)
        c[9] = m[j + 1];
        c[10] = f0 * m[j + 1];
        c[11] = j == 0 ? 0.0 : m[j + 1];
        // the E column's t_E carries dk_j / (k_j f) = nu_j (rate_consts_k)
        c[0] *= P.nu[j];
        c[3] *= P.nu[j];
        c[6] *= P.nu[j];
        c[9] *= P.nu[j];
        for (int e = 0; e < 12; e++) {
            P.kcf[j][e] = (float)c[e];
            P.kcl[j][e] = (float)(c[e] - (double)P.kcf[j][e]);
        }
    }
}

// Newton controls (pseudo-transient continuation constants are fixed).
struct NewtonCfg {
    double rtol;
    int maxit;
    // rate anchors of the step's initial state (alpha chain, power law; nullptr:
    // none): per zone kappa_j = amp_j T_a^nu_j (rows 0..nreac-1), T_a and 1/T_a
    // (rows nreac, nreac+1), written by reaction_source_kernel at U^n.  A solve
    // whose start lies within 2^-20 of T_a in temperature forms its rate
    // factors from them (rate_consts_anchor) instead of a log2 and nreac exp2.
    const double* anchor = nullptr;
};

// kappa_j(T) = kappa_j(T_a) (T / T_a)^nu_j from the zone's anchor, where
// |delta| = |T / T_a - 1| <= 2^-20 and every nu_j <= 45 (P.rate_taylor):
// T - T_a is exact (the two lie within a factor of two), delta is formed with
// the anchor's 1/T_a, ln(1 + delta) = delta - delta^2/2 + delta^3/3 (the next
// term is below 2^-82), and (1 + delta)^nu_j = exp(y), y = nu_j ln(1 + delta),
// |y| <= 45 2^-20, by exp(y) - 1 = y + y^2/2 + y^3/6 (the next term is below
// 2^-62): five FP64 operations per reaction in place of an exp2 and two products,
// and no log2.  dfac = 1/T as rate_consts_k forms it.  Returns false (nothing
// formed) where the anchor does not apply, or is not valid (T_a stored as nan).
template <int NR>
__device__ __forceinline__ bool rate_consts_anchor(const NetParams& P, double T, const double* anchor, long long N,
                                                   long long z, double* k, double& dfac) {
    if (!P.rate_taylor) return false;
    const double Ta = anchor[(long long)NR * N + z], iTa = anchor[(long long)(NR + 1) * N + z];
    const double delta = (T - Ta) * iTa;
    if (!(mag2(delta) <= mag2(0x1p-20))) return false;  // a nan delta fails
    const double L = fma(delta * delta, fma(delta, 1.0 / 3.0, -0.5), delta);
#pragma unroll
    for (int j = 0; j < NR; j++) {
        const double ka = anchor[(long long)j * N + z];
        const double y = P.nu[j] * L;
        const double p = fma(y * y, fma(y, 1.0 / 6.0, 0.5), y);
        k[j] = fma(ka, p, ka);
    }
    dfac = rcp_nr(T);
    return true;
}

// Device-side accumulators of the Newton statistics.
struct DevStats {
    unsigned long long iters_total;
    unsigned long long solves;
    unsigned long long fails;
    unsigned long long hist[64];
};

constexpr double PTC_H0 = 1.0;
constexpr double PTC_GROW = 3.0;
constexpr double PTC_SHRINK = 4.0;
constexpr double PTC_HNEWTON = 1e3;
constexpr double PTC_HMIN = 1e-12;
constexpr double XMARGIN = 1e-2;

__device__ __forceinline__ double ipow_small(double x, int c) {
    double r = 1.0;
    for (int i = 0; i < c; i++) r *= x;
    return r;
}

// k_j = a_j rho^(o_j - 1) f_j(T) and dk_j/dT for every reaction; the power
// law's T^nu_j = 2^(nu_j log2 T) by the table-driven log2 / exp2 of sdc_pow.cuh.
template <int NR>
__device__ __forceinline__ void rate_consts(const NetParams& P, double rho, double T, double* k, double* dk) {
    if (P.law == LAW_POWER) {
        const double l2T = log2_tab(T);
        const double iT = rcp_nr(T);
#pragma unroll
        for (int j = 0; j < NR; j++) {
            double rp = ipow_small(rho, P.order[j] - 1);
            double kk = P.a[j] * rp * exp2_tab(P.nu[j] * l2T);
            k[j] = kk;
            dk[j] = P.nu[j] * kk * iT;
        }
    } else {
        const double iT = rcp_nr(T);
#pragma unroll
        for (int j = 0; j < NR; j++) {
            double rp = ipow_small(rho, P.order[j] - 1);
            double kk = P.a[j] * rp * exp(-P.nu[j] * iT);
            k[j] = kk;
            dk[j] = kk * P.nu[j] * iT * iT;
        }
    }
}

// k_j only, and the factor f with dk_j/dT = nu_j k_j f (power law: f = 1/T;
// Arrhenius: f = 1/T^2): the alpha chain's matrix takes nu_j from its
// coefficients (set_chain_coefs), so the solve needs no dk_j.
// ak[j]: the prefactor of k_j = ak[j] f_j(T) (the alpha chain's amp_j).
template <int NR>
__device__ __forceinline__ void rate_consts_k(const NetParams& P, const double* ak, double T, double* k,
                                              double& dfac) {
    const double iT = rcp_nr(T);
    if (P.law == LAW_POWER) {
        const double l2T = log2_tab(T);
#pragma unroll
        for (int j = 0; j < NR; j++) k[j] = ak[j] * exp2_tab(P.nu[j] * l2T);
        dfac = iT;
    } else {
#pragma unroll
        for (int j = 0; j < NR; j++) k[j] = ak[j] * exp(-P.nu[j] * iT);
        dfac = iT * iT;
    }
}

// Per-species sums S_i = sum_j s_ij r_j and E = sum_j Q_j r_j of the rates
// r_j = k_j prod Y (R(rho X_i) = rho mass_i S_i, R(rho E) = rho E).
template <int NS, int TOPO>
__device__ __forceinline__ void source_sums(const NetParams& P, const double* k, const double* Y, double* S,
                                            double& RE) {
    constexpr int NR = NS - 1;
#pragma unroll
    for (int i = 0; i < NS; i++) S[i] = 0.0;
    RE = 0.0;
    if (TOPO == TOPO_CHAIN) {
#pragma unroll
        for (int j = 0; j < NR; j++) {
            double r = (j == 0) ? k[0] * (Y[0] * Y[0] * Y[0]) : k[j] * (Y[j] * Y[0]);
            RE += P.Q[j] * r;
            if (j == 0) {
                S[0] -= 3.0 * r;
                S[1] += r;
            } else {
                S[j] -= r;
                S[0] -= r;
                S[j + 1] += r;
            }
        }
    } else {
        for (int j = 0; j < P.nreac; j++) {
            double py = 1.0;
            if (P.r0[j] >= 0) py *= ipow_small(Y[P.r0[j]], P.c0[j]);
            if (P.r1[j] >= 0) py *= ipow_small(Y[P.r1[j]], P.c1[j]);
            double r = k[j] * py;
            RE += P.Q[j] * r;
            if (P.r0[j] >= 0) S[P.r0[j]] -= P.c0[j] * r;
            if (P.r1[j] >= 0) S[P.r1[j]] -= P.c1[j] * r;
            S[P.prod[j]] += r;
        }
    }
}

// The alpha chain's sources from kappa_j = amp_j f_j(T) and the unknowns w_X
// (rho X_i) themselves: with P_j = w_0^3 (j = 0) or w_j w_0,
//   R(rho X_i) = sum_j mass_i s_ij kappa_j P_j,   R(rho E) = sum_j Q_j kappa_j P_j
// (the density and the masses of Y_i = X_i / mass_i folded into kappa_j, the
// masses of the rows into the coefficients rs).  Rm = [R(rho E), R(rho X_i)].
template <int NS>
__device__ __forceinline__ void sources_w(const NetParams& P, const double* k, const double* w, double* Rm) {
    constexpr int NR = NS - 1;
    double r[NR];
#pragma unroll
    for (int j = 0; j < NR; j++) r[j] = (j == 0) ? k[0] * (w[0] * w[0] * w[0]) : k[j] * (w[j] * w[0]);
    double RE = P.Q[0] * r[0], S0 = P.rs[0][0] * r[0];
#pragma unroll
    for (int j = 1; j < NR; j++) {
        RE = fma(P.Q[j], r[j], RE);
        S0 = fma(P.rs[j][0], r[j], S0);
    }
    Rm[0] = RE;
    Rm[1] = S0;
#pragma unroll
    for (int i = 1; i < NS; i++) {
        // made by reaction i - 1, used by reaction i (the last species is not used)
        const double made = P.rs[i - 1][2] * r[i - 1];
        Rm[1 + i] = (i < NR) ? fma(P.rs[i][1], r[i], made) : made;
    }
}

// Reactive sources R(w) = [R(rho E), R(rho X_0..)] from the rate constants and Y.
// Alpha chain topology: j = 0 is 3 A0 -> A1, j >= 1 is A_j + A0 -> A_{j+1}.
template <int NS, int TOPO>
__device__ __forceinline__ void sources(const NetParams& P, double rho, const double* k, const double* Y,
                                        double* R) {
    double S[NS], RE;
    source_sums<NS, TOPO>(P, k, Y, S, RE);
    R[0] = rho * RE;
#pragma unroll
    for (int i = 0; i < NS; i++) R[1 + i] = rho * P.mass[i] * S[i];
}

// M = c I - dtm dR/dw, built from the rate constants (no transcendentals).
// dT/d(rho E) = (gamma-1)/rho;  dY_i/d(rho X_i) = 1/(rho mass_i).
template <int NS, int TOPO, typename MT>
__device__ __forceinline__ void build_matrix(const NetParams& P, double rho, double inv_rho, const double* ym,
                                             const double* k, const double* dk, const double* Y, double c,
                                             double dtm, MT (*M)[NS + 1]) {
    constexpr int N = NS + 1;
    constexpr int NR = NS - 1;
#pragma unroll
    for (int r = 0; r < N; r++)
#pragma unroll
        for (int q = 0; q < N; q++) M[r][q] = (r == q) ? (MT)c : (MT)0;
    const MT dTdE = (MT)(P.gm1 * inv_rho);
    const MT s = (MT)(dtm * rho);  // dtm * rho multiplies every row
    if (TOPO == TOPO_CHAIN) {
#pragma unroll
        for (int j = 0; j < NR; j++) {
            // derivatives of r_j with respect to w_E, w_X0 and w_Xj
            MT drE, drX0, drXj = (MT)0;
            if (j == 0) {
                MT y0 = (MT)Y[0];
                drE = (MT)dk[0] * (y0 * y0 * y0) * dTdE;
                drX0 = (MT)k[0] * ((MT)3 * y0 * y0) * (MT)ym[0];
            } else {
                MT y0 = (MT)Y[0], yj = (MT)Y[j];
                drE = (MT)dk[j] * (yj * y0) * dTdE;
                drXj = (MT)k[j] * y0 * (MT)ym[j];
                drX0 = (MT)k[j] * yj * (MT)ym[0];
            }
            // rows: E gets Q_j; species rows get mass_i * s_ij
            const MT qj = s * (MT)P.Q[j];
            M[0][0] -= qj * drE;
            M[0][1] -= qj * drX0;
            if (j > 0) M[0][1 + j] -= qj * drXj;
            if (j == 0) {
                const MT a0 = s * (MT)P.mass[0] * (MT)(-3.0), a1 = s * (MT)P.mass[1];
                M[1][0] -= a0 * drE;  M[1][1] -= a0 * drX0;
                M[2][0] -= a1 * drE;  M[2][1] -= a1 * drX0;
            } else {
                const MT am = s * (MT)P.mass[j] * (MT)(-1.0);
                const MT a0 = s * (MT)P.mass[0] * (MT)(-1.0);
                const MT ap = s * (MT)P.mass[j + 1];
                M[1 + j][0] -= am * drE;  M[1 + j][1] -= am * drX0;  M[1 + j][1 + j] -= am * drXj;
                M[1][0] -= a0 * drE;      M[1][1] -= a0 * drX0;      M[1][1 + j] -= a0 * drXj;
                M[2 + j][0] -= ap * drE;  M[2 + j][1] -= ap * drX0;  M[2 + j][1 + j] -= ap * drXj;
            }
        }
    } else {
        for (int j = 0; j < P.nreac; j++) {
            double py = 1.0;
            if (P.r0[j] >= 0) py *= ipow_small(Y[P.r0[j]], P.c0[j]);
            if (P.r1[j] >= 0) py *= ipow_small(Y[P.r1[j]], P.c1[j]);
            double dr[N];
#pragma unroll
            for (int q = 0; q < N; q++) dr[q] = 0.0;
            dr[0] = dk[j] * py * (P.gm1 * inv_rho);
            for (int sl = 0; sl < 2; sl++) {
                int sp = sl == 0 ? P.r0[j] : P.r1[j];
                int cn = sl == 0 ? P.c0[j] : P.c1[j];
                if (sp < 0) continue;
                double dp = cn * ipow_small(Y[sp], cn - 1);
                int o = sl == 0 ? P.r1[j] : P.r0[j];
                int oc = sl == 0 ? P.c1[j] : P.c0[j];
                if (o >= 0) dp *= ipow_small(Y[o], oc);
                dr[1 + sp] += k[j] * dp * ym[sp];
            }
            double sto[NS];
#pragma unroll
            for (int i = 0; i < NS; i++) sto[i] = 0.0;
            if (P.r0[j] >= 0) sto[P.r0[j]] -= P.c0[j];
            if (P.r1[j] >= 0) sto[P.r1[j]] -= P.c1[j];
            sto[P.prod[j]] += 1.0;
#pragma unroll
            for (int q = 0; q < N; q++) {
                M[0][q] -= (MT)(dtm * rho * P.Q[j] * dr[q]);
#pragma unroll
                for (int i = 0; i < NS; i++) M[1 + i][q] -= (MT)(dtm * rho * P.mass[i] * sto[i] * dr[q]);
            }
        }
    }
}

// The alpha chain's Newton matrix M = c I - dtm dR/dw in bordered form.  In the
// elimination order (X_1 .. X_{ns-1} | X_0, E) the chain block is lower
// bidiagonal (species i is made by reaction i-1 from species i-1 and used by
// reaction i); the alpha and energy rows and columns form the border.  Chain
// index k stands for species X_{k+1} (w index 2 + k).
template <int NS, typename MT>
struct ChainSys {
    static constexpr int NC = NS - 1;
    MT bd[NC], bs[NC];      // M[X_k][X_k], M[X_k][X_{k-1}] (bs[0] unused)
    MT uE[NC], uA[NC];      // M[X_k][E], M[X_k][X_0]
    MT vE[NC], vA[NC];      // M[E][X_k], M[X_0][X_k]
    MT dEE, dEA, dAE, dAA;  // M[E][E], M[E][X_0], M[X_0][E], M[X_0][X_0]
};

// Entries of ChainSys: M = c I - dt_m dR/dw from kappa_j = amp_j f_j(T) (the
// rates of sources_w) and w, with the per-reaction coefficients of
// set_chain_coefs.  With P_j = w_j w_0 (P_0 = w_0^3), reaction j contributes
// t_E = dt_m (gamma-1) (f / rho) kappa_j P_j to the E column (dT/d(rho E) =
// (gamma-1)/rho; nu_j is in the coefficients, f from rate_consts_k),
// t_A = dt_m kappa_j dP_j/dw_0 (without the factor 3 of j = 0) to the X_0
// column and t_J = dt_m kappa_j w_0 to the X_j column.  ws = w_1.. (the species
// part of w), dfac = f / rho.

// reaction j's coefficient e of build_chain in the matrix's working type
template <typename MT> __device__ __forceinline__ MT chain_coef(const NetParams& P, int j, int e);
template <> __device__ __forceinline__ double chain_coef<double>(const NetParams& P, int j, int e) { return P.kc[j][e]; }
template <> __device__ __forceinline__ float chain_coef<float>(const NetParams& P, int j, int e) { return P.kcf[j][e]; }
template <> __device__ __forceinline__ f2 chain_coef<f2>(const NetParams& P, int j, int e) {
    return f2(P.kcf[j][e], P.kcl[j][e]);
}

template <int NS, typename MT>
__device__ __forceinline__ void build_chain(const NetParams& P, const double* k, double dfac, const double* ws,
                                            double c, double dtm, ChainSys<NS, MT>& A) {
    constexpr int NC = NS - 1;
    constexpr int NR = NS - 1;
    const MT cm = to_mt<MT>(c);
#pragma unroll
    for (int q = 0; q < NC; q++) {
        A.bd[q] = cm;
        A.bs[q] = A.uE[q] = A.uA[q] = A.vE[q] = A.vA[q] = (MT)0;
    }
    A.dEE = A.dAA = cm;
    A.dEA = A.dAE = (MT)0;
    // t_E = t_A c0 with c0 = w_0 (gamma-1) f / rho: for j >= 1, dt_m kappa_j w_j w_0
    // (gamma-1) f / rho; for j = 0, dt_m kappa_0 w_0^3 (gamma-1) f / rho
    const MT dt_ = to_mt<MT>(dtm), c0 = to_mt<MT>(ws[0] * (P.gm1 * dfac));
    const MT y0 = to_mt<MT>(ws[0]);
#pragma unroll
    for (int j = 0; j < NR; j++) {
        auto cf = [&](int e) { return chain_coef<MT>(P, j, e); };
        if (j == 0) {
            const MT y02 = y0 * y0;
            const MT k0 = to_mt<MT>(k[0]);
            const MT t = dt_ * k0;
            const MT tA = t * y02;
            const MT tE = tA * c0;
            A.dEE = msub(A.dEE, cf(0), tE);     A.dEA = msub(A.dEA, cf(1), tA);
            A.dAE = msub(A.dAE, cf(3), tE);     A.dAA = msub(A.dAA, cf(4), tA);
            A.uE[0] = msub(A.uE[0], cf(9), tE); A.uA[0] = msub(A.uA[0], cf(10), tA);
        } else {
            const MT yj = to_mt<MT>(ws[j]), kj = to_mt<MT>(k[j]);
            const MT t = dt_ * kj;
            const MT tA = t * yj, tJ = t * y0;
            const MT tE = tA * c0;
            A.dEE = msub(A.dEE, cf(0), tE);   A.dEA = msub(A.dEA, cf(1), tA);   A.vE[j - 1] = msub(A.vE[j - 1], cf(2), tJ);
            A.dAE = msub(A.dAE, cf(3), tE);   A.dAA = msub(A.dAA, cf(4), tA);   A.vA[j - 1] = msub(A.vA[j - 1], cf(5), tJ);
            A.uE[j - 1] = msub(A.uE[j - 1], cf(6), tE);
            A.uA[j - 1] = msub(A.uA[j - 1], cf(7), tA);
            A.bd[j - 1] = msub(A.bd[j - 1], cf(8), tJ);
            A.uE[j] = msub(A.uE[j], cf(9), tE);
            A.uA[j] = msub(A.uA[j], cf(10), tA);
            A.bs[j] = msub(A.bs[j], cf(11), tJ);
        }
    }
}


// Solve M d = b for the bordered chain system (b in w order, overwritten by d).
// Gaussian elimination in the order (X_1 .. X_{ns-1} | X_0, E): at chain
// column k the pivot is the larger (ties: the first) of the row carried from
// the previous step and chain row k+1, so that the bidiagonal band keeps its
// shape and every chain step costs O(1); the border rows are eliminated along
// and the remaining 2 x 2 border block is solved with partial pivoting.  The
// solution equals the dense pivoted LU's to rounding.  Returns false on a zero
// pivot.
template <int NS, typename MT>
__device__ __forceinline__ bool chain_solve(const ChainSys<NS, MT>& A, MT* b) {
    constexpr int NC = NS - 1;
    MT pip[NC], pe[NC], puE[NC], puA[NC], pg[NC];  // pivot rows: 1/p, entry at k+1, border columns, rhs
    MT cp = A.bd[0], cuE = A.uE[0], cuA = A.uA[0], cg = b[2];  // the carried row
    MT dEE = A.dEE, dEA = A.dEA, dAE = A.dAE, dAA = A.dAA, gE = b[0], gA = b[1];
    MT wE = A.vE[0], wA = A.vA[0];  // border rows at the current column
    bool ok = true;
#pragma unroll
    for (int k = 0; k < NC; k++) {
        MT p, e, quE, quA, qg;
        if (k + 1 < NC) {
            const MT ns_ = A.bs[k + 1], nd = A.bd[k + 1], nuE = A.uE[k + 1], nuA = A.uA[k + 1], ng = b[3 + k];
            const bool sw = mag2(ns_) > mag2(cp);
            p = sw ? ns_ : cp;
            e = sw ? nd : (MT)0;
            quE = sw ? nuE : cuE;
            quA = sw ? nuA : cuA;
            qg = sw ? ng : cg;
            const MT op = sw ? cp : ns_, od = sw ? (MT)0 : nd;
            const MT ouE = sw ? cuE : nuE, ouA = sw ? cuA : nuA, og = sw ? cg : ng;
            ok = ok && nonzero(p);
            const MT ip = inv_mt(p);
            pip[k] = ip;
            const MT l = op * ip;
            cp = msub(od, l, e);
            cuE = msub(ouE, l, quE);
            cuA = msub(ouA, l, quA);
            cg = msub(og, l, qg);
        } else {
            p = cp; e = (MT)0; quE = cuE; quA = cuA; qg = cg;
            ok = ok && nonzero(p);
            pip[k] = inv_mt(p);
        }
        pe[k] = e; puE[k] = quE; puA[k] = quA; pg[k] = qg;
        const MT lE = wE * pip[k], lA = wA * pip[k];
        dEE = msub(dEE, lE, quE); dEA = msub(dEA, lE, quA); gE = msub(gE, lE, qg);
        dAE = msub(dAE, lA, quE); dAA = msub(dAA, lA, quA); gA = msub(gA, lA, qg);
        if (k + 1 < NC) {
            wE = msub(A.vE[k + 1], lE, e);
            wA = msub(A.vA[k + 1], lA, e);
        }
    }
    // 2 x 2 border block, partial pivoting
    const bool sw = mag2(dAE) > mag2(dEE);
    const MT a = sw ? dAE : dEE, bb = sw ? dAA : dEA, c2 = sw ? dEE : dAE, d2 = sw ? dEA : dAA;
    const MT r1 = sw ? gA : gE, r2 = sw ? gE : gA;
    ok = ok && nonzero(a);
    const MT ia = inv_mt(a);
    const MT l = c2 * ia;
    const MT s22 = msub(d2, l, bb);
    ok = ok && nonzero(s22);
    const MT xA = msub(r2, l, r1) * inv_mt(s22);
    const MT xE = msub(r1, bb, xA) * ia;
    b[0] = xE;
    b[1] = xA;
    MT xn = (MT)0;
#pragma unroll
    for (int k = NC - 1; k >= 0; k--) {
        const MT x = msub(msub(msub(pg[k], pe[k], xn), puE[k], xE), puA[k], xA) * pip[k];
        b[2 + k] = x;
        xn = x;
    }
    return ok;
}

// build_chain and chain_solve in one pass, for the float-pair matrix: reaction
// j's entries are formed when the elimination reaches the column that needs them
// (the chain row k+1 is complete once reaction k+2 is in, and the border entries
// at column k come from reaction k+1), so the matrix itself is never held; the
// border block accumulates reaction terms and elimination updates in whatever
// order they come (a different rounding order from build_chain + chain_solve,
// the same pivots and the same algebra).  The right-hand side G (FP64, w order)
// is converted as it is used; the step d is returned in StepType<MT>.
// Each column's record in shared memory (field f of column kk at
// piv[(f NC + kk) stride], stride = threads of the block) first holds that
// column's inputs as pairs (kappa_kk, w_kk, the chain rhs G[2 + kk]) and, once
// the elimination has read them, the pivot row (1/p, entry at kk+1, border
// columns, rhs) for the back substitution.  The elimination loop over the
// columns is not unrolled, so that its code, ten FP32 instructions per pair
// operation, stays in the instruction cache; its per-column inputs come from
// the records and the network constants from the kernel's parameter space.
template <int NS, typename MT>
__device__ __forceinline__ bool chain_build_solve(const NetParams& P, const double* k, double dfac, const double* ws,
                                                  double c, double dtm, const double* G,
                                                  typename StepType<MT>::type* d, MT* piv, int stride) {
    constexpr int NC = NS - 1;
    constexpr int NR = NS - 1;
    const MT cm = to_mt<MT>(c);
    const MT dt_ = to_mt<MT>(dtm), c0 = to_mt<MT>(ws[0] * (P.gm1 * dfac));  // t_E = t_A c0 (build_chain)
    const MT y0 = to_mt<MT>(ws[0]);
    const MT zero = (MT)0;
    auto rec = [&](int f, int kk) -> MT& { return piv[(f * NC + kk) * stride]; };
    // the inputs of every column
#pragma unroll
    for (int kk = 0; kk < NC; kk++) {
        rec(0, kk) = to_mt<MT>(k[kk]);
        rec(1, kk) = to_mt<MT>(ws[kk]);
        rec(2, kk) = to_mt<MT>(G[2 + kk]);
    }
    // border block and border right-hand side
    MT dEE = cm, dEA = zero, dAE = zero, dAA = cm;
    MT gE = to_mt<MT>(G[0]), gA = to_mt<MT>(G[1]);
    // chain rows in the making: row r (complete once reaction r+1 is in) and row r+1
    MT rbd = cm, ruE, ruA, rbs = zero;       // row r: diagonal, border columns, sub-diagonal
    MT sbs = zero, suE = zero, suA = zero;   // row r+1: the part reaction r+1 gave
    MT vEr = zero, vAr = zero;               // border rows at column r (reaction r+1)
    // reaction j >= 1's terms on the rows and columns it touches
    auto react = [&](int j, MT kj, MT yj, MT& uE_prev, MT& uA_prev, MT& bd_prev, MT& vE_prev, MT& vA_prev, MT& uE_j,
                     MT& uA_j, MT& bs_j) {
        auto cf = [&](int e) { return chain_coef<MT>(P, j, e); };
        const MT t = dt_ * kj;
        const MT tA = t * yj, tJ = t * y0;
        const MT tE = tA * c0;
        dEE = msub(dEE, cf(0), tE); dEA = msub(dEA, cf(1), tA);
        dAE = msub(dAE, cf(3), tE); dAA = msub(dAA, cf(4), tA);
        vE_prev = (MT)0 - cf(2) * tJ; vA_prev = (MT)0 - cf(5) * tJ;
        uE_prev = msub(uE_prev, cf(6), tE);
        uA_prev = msub(uA_prev, cf(7), tA);
        bd_prev = msub(bd_prev, cf(8), tJ);
        uE_j = (MT)0 - cf(9) * tE; uA_j = (MT)0 - cf(10) * tA;
        bs_j = (MT)0 - cf(11) * tJ;
    };
    {   // reactions 0 and 1: chain row 0 complete, border at column 0, row 1 begun
        auto cf = [&](int e) { return chain_coef<MT>(P, 0, e); };
        const MT y02 = y0 * y0;
        const MT k0 = rec(0, 0);
        const MT tA = dt_ * k0 * y02;
        const MT tE = tA * c0;
        dEE = msub(dEE, cf(0), tE); dEA = msub(dEA, cf(1), tA);
        dAE = msub(dAE, cf(3), tE); dAA = msub(dAA, cf(4), tA);
        ruE = (MT)0 - cf(9) * tE; ruA = (MT)0 - cf(10) * tA;
        rbs = zero;
        if (NR > 1) react(1, rec(0, 1), rec(1, 1), ruE, ruA, rbd, vEr, vAr, suE, suA, sbs);
    }
    MT cp = rbd, cuE = ruE, cuA = ruA, cg = rec(2, 0);  // the carried row
    MT wE = vEr, wA = vAr;  // border rows at the current column
    // row kk+1 (being completed) and the border entries at column kk+1
    MT nbd = cm, nuE = suE, nuA = suA, nbs = sbs;
    bool ok = true;
#pragma unroll 1
    for (int kk = 0; kk + 1 < NC; kk++) {
        // reaction kk+2 completes row kk+1 and gives the border entries at column kk+1
        MT tbd = cm, tuE = zero, tuA = zero, tbs = zero, nvE = zero, nvA = zero;
        if (kk + 2 < NR) react(kk + 2, rec(0, kk + 2), rec(1, kk + 2), nuE, nuA, nbd, nvE, nvA, tuE, tuA, tbs);
        const MT ns_ = nbs, nd = nbd, nu1 = nuE, nu2 = nuA, ng = rec(2, kk + 1);
        const bool sw = mag2(ns_) > mag2(cp);
        const MT p = sw ? ns_ : cp;
        const MT e = sw ? nd : zero;
        const MT quE = sw ? nu1 : cuE;
        const MT quA = sw ? nu2 : cuA;
        const MT qg = sw ? ng : cg;
        const MT op = sw ? cp : ns_, od = sw ? zero : nd;
        const MT ouE = sw ? cuE : nu1, ouA = sw ? cuA : nu2, og = sw ? cg : ng;
        ok = ok && nonzero(p);
        const MT ip = inv_mt(p);
        const MT l = op * ip;
        cp = msub(od, l, e);
        cuE = msub(ouE, l, quE);
        cuA = msub(ouA, l, quA);
        cg = msub(og, l, qg);
        rec(0, kk) = ip; rec(1, kk) = e; rec(2, kk) = quE; rec(3, kk) = quA; rec(4, kk) = qg;
        const MT lE = wE * ip, lA = wA * ip;
        dEE = msub(dEE, lE, quE); dEA = msub(dEA, lE, quA); gE = msub(gE, lE, qg);
        dAE = msub(dAE, lA, quE); dAA = msub(dAA, lA, quA); gA = msub(gA, lA, qg);
        wE = msub(nvE, lE, e);
        wA = msub(nvA, lA, e);
        // row kk+2 becomes the next row
        nbd = tbd; nuE = tuE; nuA = tuA; nbs = tbs;
    }
    {   // the last chain column: no row below it
        constexpr int kk = NC - 1;
        const MT p = cp;
        ok = ok && nonzero(p);
        const MT ip = inv_mt(p);
        rec(0, kk) = ip; rec(1, kk) = zero; rec(2, kk) = cuE; rec(3, kk) = cuA; rec(4, kk) = cg;
        const MT lE = wE * ip, lA = wA * ip;
        dEE = msub(dEE, lE, cuE); dEA = msub(dEA, lE, cuA); gE = msub(gE, lE, cg);
        dAE = msub(dAE, lA, cuE); dAA = msub(dAA, lA, cuA); gA = msub(gA, lA, cg);
    }
    // 2 x 2 border block, partial pivoting
    const bool sw = mag2(dAE) > mag2(dEE);
    const MT a = sw ? dAE : dEE, bb = sw ? dAA : dEA, c2 = sw ? dEE : dAE, d2 = sw ? dEA : dAA;
    const MT r1 = sw ? gA : gE, r2 = sw ? gE : gA;
    ok = ok && nonzero(a);
    const MT ia = inv_mt(a);
    const MT l = c2 * ia;
    const MT s22 = msub(d2, l, bb);
    ok = ok && nonzero(s22);
    const MT xA = msub(r2, l, r1) * inv_mt(s22);
    const MT xE = msub(r1, bb, xA) * ia;
    d[0] = step_value(xE);
    d[1] = step_value(xA);
    // back substitution, also not unrolled: each column's step (a double) goes to
    // its record's first field as raw bits, then to d
    MT xn = zero;
#pragma unroll 1
    for (int kk = NC - 1; kk >= 0; kk--) {
        const MT x = msub(msub(msub(rec(4, kk), rec(1, kk), xn), rec(2, kk), xE), rec(3, kk), xA) * rec(0, kk);
        const long long b = dbits(step_value(x));
        rec(0, kk) = MT(__int_as_float((int)b), __int_as_float((int)(b >> 32)));
        xn = x;
    }
#pragma unroll
    for (int kk = 0; kk < NC; kk++) {
        const MT v = rec(0, kk);
        d[2 + kk] = bitsd(((long long)__float_as_int(v.lo) << 32) | (long long)(unsigned)__float_as_int(v.hi));
    }
    return ok;
}

// In-place LU with partial pivoting (largest |entry|, ties to the lowest row)
// and solve of M d = b; b is overwritten with d.  Row exchanges are done with
// predicated selects so that M stays in registers.  Returns false on a zero pivot.
template <int N, typename MT, typename VT>
__device__ __forceinline__ bool lu_solve(MT (*M)[N], VT* b) {
    MT inv_piv[N];
#pragma unroll
    for (int kc = 0; kc < N; kc++) {
        // pivot search (|x| compared as shifted bit patterns, mag2: they order like the values)
        int piv = kc;
        {
            auto best = mag2(M[kc][kc]);
#pragma unroll
            for (int i = kc + 1; i < N; i++) {
                const auto v = mag2(M[i][kc]);
                if (v > best) { best = v; piv = i; }
            }
            if (best == 0) return false;
        }
        // exchange rows kc and piv
#pragma unroll
        for (int i = kc + 1; i < N; i++) {
            const bool sw = (i == piv);
#pragma unroll
            for (int q = kc; q < N; q++) {
                MT a = M[kc][q], bq = M[i][q];
                M[kc][q] = sw ? bq : a;
                M[i][q] = sw ? a : bq;
            }
            VT x = b[kc], y = b[i];
            b[kc] = sw ? y : x;
            b[i] = sw ? x : y;
        }
        const MT ip = (sizeof(MT) == 8) ? (MT)rcp_nr((double)M[kc][kc]) : (MT)1 / M[kc][kc];
        inv_piv[kc] = ip;
#pragma unroll
        for (int i = kc + 1; i < N; i++) {
            const MT l = M[i][kc] * ip;
#pragma unroll
            for (int q = kc + 1; q < N; q++) M[i][q] -= l * M[kc][q];
            b[i] -= (VT)l * b[kc];
        }
    }
#pragma unroll
    for (int i = N - 1; i >= 0; i--) {
        VT s = b[i];
#pragma unroll
        for (int q = i + 1; q < N; q++) s -= (VT)M[i][q] * b[q];
        b[i] = s * (VT)inv_piv[i];
    }
    return true;
}

}  // namespace sdcd
