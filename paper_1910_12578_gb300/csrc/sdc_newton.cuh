// sdc_newton.cuh -- per-zone implicit reaction update of Eq. sdc:general
// (paper section 2: the reactive part of the node update is implicit in the new state):
//   G(w) = w - dt_m R(w; rho, rho u) - rhs_w = 0,   w = (rho E, rho X_i)
// solved by Newton iteration on M = c I - dt_m dR/dw (c = 1), globalised by
// pseudo-transient continuation (c = 1 + 1/h):
//   start in Newton mode; a trial is admissible when T > 0 (finite) and, when
//   every X_i(rhs) >= -0.01, every X_i >= min(0, X_i(rhs), X_i(start)) - 0.01
//   (no floor for an rhs pushed further negative); a Newton trial that is not
//   admissible or raises the scaled residual switches to pseudo mode (h = 1);
//   an admissible pseudo trial is taken and h *= 3, a rejected one h /= 4;
//   h >= 1e3 returns to Newton mode; converged when an admissible Newton step
//   has max(|d(rho E)|/|rho E|, max_i |d(rho X_i)|/rho) <= rtol (taken even if
//   the residual grew by round-off at the root).
// One thread owns one zone; the matrix lives in registers as MT (double: FP64
// path; float: FP32 Jacobian / LU with FP64 residual and update, so that Newton
// acts as iterative refinement; f2, the alpha chain only: the same with the
// matrix in float pairs on the FP32 pipe, whose step is accurate to about 2^-44
// relative, so the iteration keeps the FP64 path's count of steps): dense with a
// pivoted LU for a general network,
// in the bordered bidiagonal form of the alpha chain (build_chain, chain_solve)
// for the chain.
#pragma once
#include <type_traits>

#include "sdc_dev.cuh"

namespace sdcd {

// Dynamic shared memory of the one-zone-per-thread kernels: the float-pair
// solve's pivot rows (pair_pivot_bytes per block; none for the other types),
// then every thread's composition floors (NS doubles, stride blockDim.x).
extern __shared__ double newton_smem[];

template <int NS, typename MT>
__host__ __device__ constexpr size_t pair_pivot_bytes(int block) {
    return std::is_same<MT, f2>::value ? (size_t)5 * (NS - 1) * sizeof(f2) * (size_t)block : 0;
}

template <int NS, typename MT>
__host__ __device__ constexpr size_t newton_smem_bytes(int block) {
    return pair_pivot_bytes<NS, MT>(block) + (size_t)NS * sizeof(double) * (size_t)block;
}

// this thread's first composition floor (the next at + blockDim.x, ...)
template <int NS, typename MT>
__device__ __forceinline__ double* newton_floor_smem() {
    return newton_smem + pair_pivot_bytes<NS, MT>((int)blockDim.x) / sizeof(double) + threadIdx.x;
}

template <int NS, int TOPO>
struct ZoneEval {
    static constexpr int N = NS + 1;
    static constexpr int NR = NS - 1;
};

// Evaluate T, rate constants, Y and the residual at state w, in the order of
// operations of the definition, G = w - dt_m R(w) - rhs_w, and its scaled norm
// times rho^2, phi = (G_E rho/|rhs_E|)^2 + sum_i G_i^2 (the solve only compares
// norms of one zone, so the common factor 1/rho^2 of the scaled norm
// (G_E/|rhs_E|)^2 + sum_i (G_i/rho)^2 is left out).  For the alpha chain only
// kappa_j = amp_j f_j(T), whose products with the unknowns are the sources
// (sources_w: no Y_i, no density), and the factor f of dkappa_j/dT =
// nu_j kappa_j f are formed (the matrix takes nu_j from its coefficients);
// otherwise k_j, dk_j and Y_i.
// Returns false when T is not positive and finite.
// The order of doubles as signed integers (negative patterns reversed), for
// comparisons on the integer pipe; -0 sorts below +0 and a nan above +inf.
__device__ __forceinline__ long long ordered_bits(double x) {
    const long long b = dbits(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}

// T > 0 and finite, on the bit pattern (integer pipe): a positive sign with a
// nonzero pattern and an exponent field below 0x7ff (nan and inf excluded)
__device__ __forceinline__ bool positive_finite(double T) {
    const long long b = dbits(T);
    return b > 0 && (b >> 52) < 0x7ff;
}

// The scaled norm phi of a residual G (see eval_state).
template <int N>
__device__ __forceinline__ double residual_norm(const double* G, double wE) {
    const double gE = G[0] * wE;
    double s = gE * gE;
#pragma unroll
    for (int r = 1; r < N; r++) s = fma(G[r], G[r], s);
    return s;
}

// eval_at_T: the same at a state whose temperature T is known to be positive
// and finite (formed by the caller as P.gm1 * (w[0] - ke) * inv_rho).  With
// PHI false the norm is left for later (have_phi false) where the exponents of
// G and wE alone show it finite: every |G_r| and |G_0 wE| below 2^500 bounds
// it by 2^1004 (integer pipe); otherwise it is formed as with PHI.
// With anchor (the step's rate anchors, see NewtonCfg) the alpha chain's rate
// factors come from zone z's anchor where it applies.
template <int NS, int TOPO, bool PHI = true>
__device__ __forceinline__ bool eval_at_T(const NetParams& P, double rho, double T, const double* ym,
                                          const double* w, const double* rw, double dtm, double wE, double* k,
                                          double* dk, double& dfac, double* Y, double* G, double& phi,
                                          bool* have_phi = nullptr, const double* anchor = nullptr, long long NZ = 0,
                                          long long z = 0) {
    constexpr int N = NS + 1;
    constexpr int NR = NS - 1;
    // G = w - dt_m R(w) - rw, formed as (w - rw) - dt_m R
    if constexpr (TOPO == TOPO_CHAIN) {
        // kappa_j = amp_j f_j(T) with the masses and density folded in: the
        // sources are products of the unknowns themselves (no Y_i)
        double R[N];
        if (!(anchor && rate_consts_anchor<NR>(P, T, anchor, NZ, z, k, dfac))) rate_consts_k<NR>(P, P.amp, T, k, dfac);
        sources_w<NS>(P, k, w + 1, R);
#pragma unroll
        for (int r = 0; r < N; r++) G[r] = fma(-dtm, R[r], w[r] - rw[r]);
    } else {
        // R(rho E) = rho RE, R(rho X_i) = rho mass_i S_i: (w - rw) - (dt_m rho) (mass_i S_i)
        double S[NS], RE;
        rate_consts<NR>(P, rho, T, k, dk);
#pragma unroll
        for (int i = 0; i < NS; i++) Y[i] = w[1 + i] * ym[i];
        source_sums<NS, TOPO>(P, k, Y, S, RE);
        const double dr = dtm * rho;
        G[0] = fma(-dr, RE, w[0] - rw[0]);
#pragma unroll
        for (int i = 0; i < NS; i++) G[1 + i] = fma(-dr, P.mass[i] * S[i], w[1 + i] - rw[1 + i]);
    }
    if constexpr (!PHI) {
        // biased exponents: |x| < 2^(e - 1022); finite G_r with e <= 1522 are below
        // 2^500, and G_0 wE is when e(G_0) + e(wE) <= 2544
        auto bexp = [](double x) { return (int)((dbits(x) >> 52) & 0x7ff); };
        bool small = bexp(G[0]) + bexp(wE) <= 2544;
#pragma unroll
        for (int r = 0; r < N; r++) small = small && bexp(G[r]) <= 1522;
        if (small) {
            *have_phi = false;
            return true;
        }
        *have_phi = true;
    }
    const double s = residual_norm<N>(G, wE);
    phi = s;
    return (dbits(s) >> 52) < 0x7ff;  // s >= 0: finite (nan and inf have the full exponent)
}

template <int NS, int TOPO>
__device__ __forceinline__ bool eval_state(const NetParams& P, double rho, double inv_rho, double ke,
                                           const double* ym, const double* w, const double* rw, double dtm,
                                           double wE, double* k, double* dk, double& dfac, double* Y, double* G,
                                           double& phi) {
    const double T = P.gm1 * (w[0] - ke) * inv_rho;
    if (!positive_finite(T)) return false;
    return eval_at_T<NS, TOPO>(P, rho, T, ym, w, rw, dtm, wE, k, dk, dfac, Y, G, phi);
}

// Register-resident state of one zone's solve.  The reactive part of the rhs
// stays in global memory (rwp, stride rws; needed again only where a trial is
// evaluated in full) and the composition floors in shared memory (lop, stride
// los), so that neither holds registers through the solve.
template <int NS>
struct ZoneState {
    static constexpr int N = NS + 1;
    static constexpr int NR = NS - 1;
    double rho, inv_rho, ke, wE, phi, h, dfac;
    double ym[NS], w[N], G[N], k[NR], dk[NR], Y[NS];  // ym, dk, Y: general networks
    const double* rwp;
    long long rws;
    double* lop;
    int los;
    int iters, status;
    bool newton, have_k, done;
    bool have_phi;  // phi holds the norm of G (at the start it is formed only when a decision needs it)
    bool r_final;   // G holds R at the solution (set by the stop test's last step)
};

// Set up a zone: rw = reactive part of the rhs (S.rwp points at it in global
// memory, S.lop at the zone's floors in shared memory), w = the (density-rescaled)
// guess; inv_rho = 1/rho, ke = |rho u|^2 / (2 rho) of the rhs, mr = -0.01 rho,
// Tw = the temperature of w when the caller has formed it and found it
// positive and finite, else 0.  Evaluates the residual at the start.
template <int NS, int TOPO>
__device__ __forceinline__ void zone_init(ZoneState<NS>& S, const NetParams& P, const double* rw, double rho,
                                          double inv_rho, double ke, double mr, double Tw, double dtm,
                                          const double* anchor = nullptr, long long NZ = 0, long long z = 0) {
    constexpr int N = NS + 1;
    S.rho = rho;
    S.inv_rho = inv_rho;
    S.ke = ke;
    if constexpr (TOPO != TOPO_CHAIN) {
#pragma unroll
        for (int i = 0; i < NS; i++) S.ym[i] = S.inv_rho * P.inv_mass[i];
    }
    S.wE = rho * rcp_nr(fabs(rw[0]));  // rho / |rhs_E|
    // a start without a positive temperature is replaced by rhs
    double T = Tw;
    if (!positive_finite(T)) {
        T = P.gm1 * (S.w[0] - S.ke) * S.inv_rho;
        if (!positive_finite(T)) {
#pragma unroll
            for (int r = 0; r < N; r++) S.w[r] = rw[r];
            T = P.gm1 * (S.w[0] - S.ke) * S.inv_rho;
        }
    }
    // the floor applies when the rhs is physical (every X_i >= -0.01), and is
    // min(0, X_i(rhs), X_i(start)) - 0.01; both are taken in units of rho X_i
    // (rho > 0): rho X_i(rhs) >= -0.01 rho, and min(0, rw_i, w_i) - 0.01 rho,
    // compared and selected on the integer pipe
    const long long omr = ordered_bits(mr);
    bool physical = true;
#pragma unroll
    for (int i = 0; i < NS; i++) physical = physical && (ordered_bits(rw[1 + i]) >= omr);
#pragma unroll
    for (int i = 0; i < NS; i++) {
        const double x = rw[1 + i], xg = S.w[1 + i];
        double lo = ordered_bits(x) < 0 ? x : 0.0;
        lo = ordered_bits(xg) < ordered_bits(lo) ? xg : lo;
        S.lop[i * S.los] = physical ? lo + mr : -INFINITY;  // as a bound on rho X_i
    }
    S.iters = 0;
    S.status = ZONE_MAXIT;
    S.newton = true;
    S.r_final = false;
    S.h = PTC_H0;
    S.have_k = positive_finite(T) && eval_at_T<NS, TOPO, false>(P, rho, T, S.ym, S.w, rw, dtm, S.wE, S.k, S.dk,
                                                                S.dfac, S.Y, S.G, S.phi, &S.have_phi, anchor, NZ, z);
    S.done = !S.have_k;
    if (!S.have_k) S.status = ZONE_NONPHYSICAL;
}

// The stop test: max(|d(rho E)|/|rho E|, max_i |d(rho X_i)|/rho) <= rtol at the trial.
template <int NS, typename MT>
__device__ __forceinline__ bool newton_step_small(const ZoneState<NS>& S, const NewtonCfg& cfg, const MT* dv,
                                                  const double* tr) {
    // |dv_0| <= rtol |tr_0| on the bit patterns (rtol > 0: |rtol tr_0| is the rounded
    // rtol |tr_0|; a nan step fails)
    bool small = mag2(from_mt(dv[0])) <= mag2(cfg.rtol * tr[0]);
    const double tol_x = cfg.rtol * S.rho;
    if constexpr (sizeof(MT) == 8) {
        // |dv_i| <= tol_x on the integer pipe (mag2 orders like |x|; a nan step fails)
        const unsigned long long mt = mag2(tol_x);
#pragma unroll
        for (int i = 0; i < NS; i++) small = small && (mag2((double)dv[1 + i]) <= mt);
    } else {
        // a float |dv_i| is <= tol_x exactly when it is <= the largest float not
        // above tol_x; compared on the integer pipe (a nan step fails)
        const unsigned int mt = mag2(__double2float_rd(tol_x));
#pragma unroll
        for (int i = 0; i < NS; i++) small = small && (mag2(dv[1 + i]) <= mt);
    }
    return small;
}

// One pass of the solve (one linear solve); sets done and status at the end.
template <int NS, int TOPO, typename MT>
__device__ __forceinline__ void zone_iterate(ZoneState<NS>& S, const NetParams& P, const NewtonCfg& cfg, double dtm) {
    constexpr int N = NS + 1;
    constexpr int NR = NS - 1;
    S.iters++;
    const double c = S.newton ? 1.0 : 1.0 + rcp_nr(S.h);
    // the step as tested and applied (a float pair summed into a double once)
    using ST = typename StepType<MT>::type;
    ST ds[N];
    bool solved;
    if constexpr (TOPO == TOPO_CHAIN && std::is_same<MT, f2>::value) {
        // float pairs: the matrix formed as the elimination reaches it
        solved = chain_build_solve<NS, MT>(P, S.k, S.dfac * S.inv_rho, S.w + 1, c, dtm, S.G, ds,
                                           reinterpret_cast<f2*>(newton_smem) + threadIdx.x, (int)blockDim.x);
    } else {
        MT dv[N];
#pragma unroll
        for (int r = 0; r < N; r++) dv[r] = to_mt<MT>(S.G[r]);
        if constexpr (TOPO == TOPO_CHAIN) {
            // the chain's sparsity: bordered bidiagonal system, O(n) elimination
            ChainSys<NS, MT> A;
            build_chain<NS, MT>(P, S.k, S.dfac * S.inv_rho, S.w + 1, c, dtm, A);
            solved = chain_solve<NS, MT>(A, dv);
        } else {
            MT M[N][N];
            build_matrix<NS, TOPO, MT>(P, S.rho, S.inv_rho, S.ym, S.k, S.dk, S.Y, c, dtm, M);
            solved = lu_solve<N, MT, MT>(M, dv);
        }
#pragma unroll
        for (int r = 0; r < N; r++) ds[r] = step_value(dv[r]);
    }
    if (!solved) {
        S.status = ZONE_SINGULAR;
        S.done = true;
        return;
    }
    double tr[N];
#pragma unroll
    for (int r = 0; r < N; r++) tr[r] = S.w[r] - from_mt(ds[r]);
    // admissible: every rho X_i at or above its floor (the floor is -inf or a
    // nonzero value, so the two zeros never meet; a nan trial passes here and
    // fails the evaluation below, as it fails this test in plain compares)
    bool ok = true;
#pragma unroll
    for (int i = 0; i < NS; i++) ok = ok && (ordered_bits(tr[1 + i]) >= ordered_bits(S.lop[i * S.los]));
    if (S.newton && ok && newton_step_small<NS, ST>(S, cfg, ds, tr)) {
        // The step meets the stop test, so an admissible trial (T positive and
        // finite, R finite) is the solution: only R at the trial is needed, not
        // the residual, its norm or the matrix's factor f.  Otherwise the full
        // evaluation below takes the decision.
        double kf[NR], dkf[NR], Yf[NS], Rf[N];
        bool have_rates = false;
        if constexpr (TOPO == TOPO_CHAIN) {
            // delta = (T - T_w) / T_w from the energy step (tr_0 - w_0 is exact:
            // the two lie within a factor of two; dfac = 1 / T_w for the power
            // law).  Where |delta| <= 2^-32, kappa_j(T) = kappa_j(T_w) (1 + nu_j
            // delta) to within the rounding of kappa: the next term of
            // (1 + delta)^nu_j, nu_j (nu_j - 1) delta^2 / 2, is below 2^-55 for
            // nu_j <= 45 (P.rate_taylor).  There T is positive and finite: T_w is,
            // and T_w <= 2^1021 (dfac >= 2^-1021, its exponent field >= 2), so T
            // within 2^-31 of it stays below the overflow threshold.
            const double delta = P.gm1 * (tr[0] - S.w[0]) * S.inv_rho * S.dfac;
            if (P.rate_taylor && mag2(delta) <= mag2(0x1p-32) && (dbits(S.dfac) >> 52) >= 2) {
#pragma unroll
                for (int j = 0; j < NR; j++) kf[j] = fma(S.k[j], P.nu[j] * delta, S.k[j]);
                have_rates = true;
            }
        }
        if (!have_rates) {
            // else the rate factors are evaluated at a positive, finite T
            const double T = P.gm1 * (tr[0] - S.ke) * S.inv_rho;
            if (positive_finite(T)) {
                if constexpr (TOPO == TOPO_CHAIN) {
                    double dff;
                    rate_consts_k<NR>(P, P.amp, T, kf, dff);
                } else {
                    rate_consts<NR>(P, S.rho, T, kf, dkf);
                }
                have_rates = true;
            }
        }
        if (have_rates) {
            if constexpr (TOPO == TOPO_CHAIN) {
                sources_w<NS>(P, kf, tr + 1, Rf);
            } else {
#pragma unroll
                for (int i = 0; i < NS; i++) Yf[i] = tr[1 + i] * S.ym[i];
                sources<NS, TOPO>(P, S.rho, kf, Yf, Rf);
            }
            bool finite = true;
#pragma unroll
            for (int r = 0; r < N; r++) finite = finite && (((dbits(Rf[r]) >> 52) & 0x7ff) != 0x7ff);
            if (finite) {
#pragma unroll
                for (int r = 0; r < N; r++) { S.w[r] = tr[r]; S.G[r] = Rf[r]; }
                S.r_final = true;
                S.status = ZONE_OK;
                S.done = true;
                return;
            }
        }
    }
    double kt[NR], dkt[NR], Yt[NS], Gt[N];
    double phit = 0.0, dfact = 0.0;
    if (ok) {
        double rwt[N];
#pragma unroll
        for (int r = 0; r < N; r++) rwt[r] = __ldg(S.rwp + r * S.rws);
        ok = eval_state<NS, TOPO>(P, S.rho, S.inv_rho, S.ke, S.ym, tr, rwt, dtm, S.wE, kt, dkt, dfact, Yt, Gt, phit);
    }
    // an admissible Newton step that meets the stop test converges even if the
    // residual grew by round-off at the root
    const bool small = S.newton && ok && newton_step_small<NS, ST>(S, cfg, ds, tr);
    if (!S.have_phi) {
        S.phi = residual_norm<N>(S.G, S.wE);
        S.have_phi = true;
    }
    // phit and phi are finite and non-negative where compared: ordered as integers
    if (S.newton && !small && (!ok || ordered_bits(phit) > ordered_bits(S.phi))) {
        S.newton = false;
        S.h = PTC_H0;
    } else if (!ok) {
        S.h /= PTC_SHRINK;
        if (S.h < PTC_HMIN) {
            S.status = ZONE_NONPHYSICAL;
            S.done = true;
            return;
        }
    } else {
#pragma unroll
        for (int r = 0; r < N; r++) { S.w[r] = tr[r]; S.G[r] = Gt[r]; }
#pragma unroll
        for (int j = 0; j < NR; j++) S.k[j] = kt[j];
        if constexpr (TOPO == TOPO_CHAIN) {
            S.dfac = dfact;
        } else {
#pragma unroll
            for (int j = 0; j < NR; j++) S.dk[j] = dkt[j];
#pragma unroll
            for (int i = 0; i < NS; i++) S.Y[i] = Yt[i];
        }
        S.phi = phit;
        if (S.newton) {
            if (small) {
                S.status = ZONE_OK;
                S.done = true;
                return;
            }
        } else {
            S.h *= PTC_GROW;
            if (S.h >= PTC_HNEWTON) S.newton = true;
        }
    }
    if (S.iters >= cfg.maxit) S.done = true;  // status stays ZONE_MAXIT
}

// Reactive source at the final state (from its cached rate constants).
template <int NS, int TOPO>
__device__ __forceinline__ void zone_source(const ZoneState<NS>& S, const NetParams& P, double* Rout) {
    constexpr int N = NS + 1;
    constexpr int NR = NS - 1;
    if (S.r_final) {
#pragma unroll
        for (int r = 0; r < N; r++) Rout[r] = S.G[r];
    } else if (S.have_k) {
        if constexpr (TOPO == TOPO_CHAIN) sources_w<NS>(P, S.k, S.w + 1, Rout);
        else sources<NS, TOPO>(P, S.rho, S.k, S.Y, Rout);
    } else {
        const double T = P.gm1 * (S.w[0] - S.ke) * S.inv_rho;
        double kf[NR], dkf[NR], Yf[NS];
        if constexpr (TOPO == TOPO_CHAIN) {
            double dff;
            rate_consts_k<NR>(P, P.amp, T, kf, dff);
            sources_w<NS>(P, kf, S.w + 1, Rout);
        } else {
            rate_consts<NR>(P, S.rho, T, kf, dkf);
#pragma unroll
            for (int i = 0; i < NS; i++) Yf[i] = S.w[1 + i] * S.ym[i];
            sources<NS, TOPO>(P, S.rho, kf, Yf, Rout);
        }
    }
}

}  // namespace sdcd
