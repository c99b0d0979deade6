// sdc_newton.cuh -- per-zone implicit reaction update of Eq. sdc:general
// (paper section 2: "an implicit equation for the new state"):
//   G(w) = w - dt_m R(w; rho, rho u) - rhs_w = 0,   w = (rho E, rho X_i)
// solved by Newton iteration on M = c I - dt_m dR/dw (c = 1), globalised by
// pseudo-transient continuation (c = 1 + 1/h):
//   start in Newton mode; a trial is admissible when T > 0 (finite) and every
//   X_i >= min(0, X_i(rhs), X_i(start)) - 0.01; a Newton trial that is not
//   admissible or raises the scaled residual switches to pseudo mode (h = 1);
//   an admissible pseudo trial is taken and h *= 3, a rejected one h /= 4;
//   h >= 1e3 returns to Newton mode; converged when a taken Newton step has
//   max(|d(rho E)|/|rho E|, max_i |d(rho X_i)|/rho) <= rtol.
// One thread owns one zone; the dense matrix lives in registers as MT
// (double: FP64 path; float: FP32 Jacobian / LU with FP64 residual and update,
// so that Newton acts as iterative refinement).
#pragma once
#include "sdc_dev.cuh"

namespace sdcd {

template <int NS, int TOPO>
struct ZoneEval {
    static constexpr int N = NS + 1;
    static constexpr int NR = NS - 1;
};

// Evaluate T, rate constants, Y and the residual at state w.
// Returns false when T is not positive and finite.
template <int NS, int TOPO>
__device__ __forceinline__ bool eval_state(const NetParams& P, double rho, double inv_rho, double ke,
                                           const double* ym, const double* w, const double* rw, double dtm,
                                           double sE_inv, double* k, double* dk, double* Y, double* G,
                                           double& phi) {
    constexpr int N = NS + 1;
    constexpr int NR = NS - 1;
    const double T = P.gm1 * (w[0] - ke) * inv_rho;
    if (!(T > 0.0 && T < INFINITY)) return false;
    rate_consts<NR>(P, rho, T, k, dk);
#pragma unroll
    for (int i = 0; i < NS; i++) Y[i] = w[1 + i] * ym[i];
    double R[N];
    sources<NS, TOPO>(P, rho, k, Y, R);
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < N; r++) {
        G[r] = w[r] - dtm * R[r] - rw[r];
        const double g = r == 0 ? G[r] * sE_inv : G[r] * inv_rho;
        s += g * g;
    }
    phi = s;
    return s < INFINITY;
}

// Solve one zone.  On entry w holds the (density-rescaled) guess; on exit the
// last taken iterate, R its reactive source.  Returns a ZONE_* code.
template <int NS, int TOPO, typename MT>
__device__ __forceinline__ int newton_zone(const NetParams& P, const NewtonCfg& cfg, double rho, double m2,
                                           const double* rw, double dtm, double* w, double* Rout, int& iters) {
    constexpr int N = NS + 1;
    constexpr int NR = NS - 1;
    const double inv_rho = rcp_nr(rho);
    const double ke = 0.5 * m2 * inv_rho;
    double ym[NS];
#pragma unroll
    for (int i = 0; i < NS; i++) ym[i] = inv_rho * P.inv_mass[i];
    const double sE_inv = rcp_nr(fabs(rw[0]));

    // a start without a positive temperature is replaced by rhs
    {
        const double Tg = P.gm1 * (w[0] - ke) * inv_rho;
        if (!(Tg > 0.0 && Tg < INFINITY)) {
#pragma unroll
            for (int r = 0; r < N; r++) w[r] = rw[r];
        }
    }
    double lower[NS];
#pragma unroll
    for (int i = 0; i < NS; i++) {
        const double x = rw[1 + i] * inv_rho, xg = w[1 + i] * inv_rho;
        double lo = x < 0.0 ? x : 0.0;
        lo = xg < lo ? xg : lo;
        lower[i] = (lo - XMARGIN) * rho;  // as a bound on rho X_i
    }
    double k[NR], dk[NR], Y[NS], G[N];
    double phi;
    int status = ZONE_MAXIT;
    iters = 0;
    const bool have_k = eval_state<NS, TOPO>(P, rho, inv_rho, ke, ym, w, rw, dtm, sE_inv, k, dk, Y, G, phi);
    if (!have_k) {
        status = ZONE_NONPHYSICAL;
    } else {
        bool newton = true;
        double h = PTC_H0;
        int it;
        for (it = 1; it <= cfg.maxit; it++) {
            const double c = newton ? 1.0 : 1.0 + rcp_nr(h);
            MT M[N][N];
            build_matrix<NS, TOPO, MT>(P, rho, inv_rho, ym, k, dk, Y, c, dtm, M);
            MT dv[N];
#pragma unroll
            for (int r = 0; r < N; r++) dv[r] = (MT)G[r];
            if (!lu_solve<N, MT, MT>(M, dv)) { status = ZONE_SINGULAR; break; }
            double tr[N];
#pragma unroll
            for (int r = 0; r < N; r++) tr[r] = w[r] - (double)dv[r];
            bool ok = true;
#pragma unroll
            for (int i = 0; i < NS; i++) ok = ok && (tr[1 + i] >= lower[i]);
            double kt[NR], dkt[NR], Yt[NS], Gt[N];
            double phit = 0.0;
            if (ok) ok = eval_state<NS, TOPO>(P, rho, inv_rho, ke, ym, tr, rw, dtm, sE_inv, kt, dkt, Yt, Gt, phit);
            if (newton && (!ok || phit > phi)) {
                newton = false;
                h = PTC_H0;
                continue;
            }
            if (!ok) {
                h /= PTC_SHRINK;
                if (h < PTC_HMIN) { status = ZONE_NONPHYSICAL; break; }
                continue;
            }
#pragma unroll
            for (int r = 0; r < N; r++) { w[r] = tr[r]; G[r] = Gt[r]; }
#pragma unroll
            for (int j = 0; j < NR; j++) { k[j] = kt[j]; dk[j] = dkt[j]; }
#pragma unroll
            for (int i = 0; i < NS; i++) Y[i] = Yt[i];
            phi = phit;
            if (newton) {
                bool conv = fabs((double)dv[0]) <= cfg.rtol * fabs(w[0]);
                const double tol_x = cfg.rtol * rho;
#pragma unroll
                for (int i = 0; i < NS; i++) conv = conv && (fabs((double)dv[1 + i]) <= tol_x);
                if (conv) { status = ZONE_OK; break; }
            } else {
                h *= PTC_GROW;
                if (h >= PTC_HNEWTON) newton = true;
            }
        }
        iters = it > cfg.maxit ? cfg.maxit : it;
    }
    // reactive source at the final state (from its cached rate constants)
    if (have_k) {
        sources<NS, TOPO>(P, rho, k, Y, Rout);
    } else {
        const double T = P.gm1 * (w[0] - ke) * inv_rho;
        double kf[NR], dkf[NR], Yf[NS];
        rate_consts<NR>(P, rho, T, kf, dkf);
#pragma unroll
        for (int i = 0; i < NS; i++) Yf[i] = w[1 + i] * ym[i];
        sources<NS, TOPO>(P, rho, kf, Yf, Rout);
    }
    return status;
}

}  // namespace sdcd
