// sdc_dev.cuh -- device-side building blocks of the SDC hot path on sm_103a:
// network parameters, gamma-law EOS, rate constants, reactive sources and
// their Jacobian, and the dense pivoted LU of the implicit reaction update.
//
// Paper: arXiv:1910.12578, section 2 (Eq. 1, Eq. sdc:general).  The network,
// EOS and Newton globalisation are the readings stated in sdc.h / the design
// notes: r_j = a_j rho^(o_j-1) f_j(T) prod Y^cnt, p = rho T, e = T/(gamma-1).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sdc_fastmath.cuh"

#define SDCD_MAXS 16
#define SDCD_MAXR 16

namespace sdcd {

enum { TOPO_GENERIC = 0, TOPO_CHAIN = 1 };
enum { LAW_POWER = 0, LAW_ARRHENIUS = 1 };
enum { ZONE_OK = 0, ZONE_MAXIT = 1, ZONE_NONPHYSICAL = 2, ZONE_SINGULAR = 3 };

// Network and gas constants, passed by value to every kernel.
struct NetParams {
    int nspec, nreac, law, topo;
    double gm1;                          // gamma - 1
    double gamma;
    double mass[SDCD_MAXS];
    double inv_mass[SDCD_MAXS];
    double a[SDCD_MAXR], nu[SDCD_MAXR], Q[SDCD_MAXR];
    int r0[SDCD_MAXR], c0[SDCD_MAXR], r1[SDCD_MAXR], c1[SDCD_MAXR], prod[SDCD_MAXR];
    int order[SDCD_MAXR];                // sum of reactant multiplicities
};

// Newton controls (pseudo-transient continuation constants are fixed).
struct NewtonCfg {
    double rtol;
    int maxit;
};

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

// k_j = a_j rho^(o_j - 1) f_j(T) and dk_j/dT for every reaction.
template <int NR>
__device__ __forceinline__ void rate_consts(const NetParams& P, double rho, double T, double* k, double* dk) {
    if (P.law == LAW_POWER) {
        const double lT = log(T);
        const double iT = rcp_nr(T);
#pragma unroll
        for (int j = 0; j < NR; j++) {
            double rp = ipow_small(rho, P.order[j] - 1);
            double kk = P.a[j] * rp * exp(P.nu[j] * lT);
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

// Reactive sources R(w) = [R(rho E), R(rho X_0..)] from the rate constants and Y.
// Alpha chain topology: j = 0 is 3 A0 -> A1, j >= 1 is A_j + A0 -> A_{j+1}.
template <int NS, int TOPO>
__device__ __forceinline__ void sources(const NetParams& P, double rho, const double* k, const double* Y,
                                        double* R) {
    constexpr int NR = NS - 1;
    double S[NS];
#pragma unroll
    for (int i = 0; i < NS; i++) S[i] = 0.0;
    double RE = 0.0;
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

// In-place LU with partial pivoting (largest |entry|, ties to the lowest row)
// and solve of M d = b; b is overwritten with d.  Row exchanges are done with
// predicated selects so that M stays in registers.  Returns false on a zero pivot.
template <int N, typename MT, typename VT>
__device__ __forceinline__ bool lu_solve(MT (*M)[N], VT* b) {
    MT inv_piv[N];
#pragma unroll
    for (int kc = 0; kc < N; kc++) {
        // pivot search (|x| compared as bit patterns: they order like the values)
        int piv = kc;
        if (sizeof(MT) == 8) {
            long long best = __double_as_longlong((double)M[kc][kc]) & ABS_MASK;
#pragma unroll
            for (int i = kc + 1; i < N; i++) {
                const long long v = __double_as_longlong((double)M[i][kc]) & ABS_MASK;
                if (v > best) { best = v; piv = i; }
            }
            if (best == 0) return false;
        } else {
            int best = __float_as_int((float)M[kc][kc]) & 0x7fffffff;
#pragma unroll
            for (int i = kc + 1; i < N; i++) {
                const int v = __float_as_int((float)M[i][kc]) & 0x7fffffff;
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
