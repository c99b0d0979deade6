// sdc_newton_group.cuh -- the implicit reaction update of Eq. sdc:general
// (paper section 2) with a group of L lanes per zone, for networks whose
// dense Jacobian does not fit one thread's registers (14 x 14 for the
// 13-species chain).
//
// Same algorithm, step for step, as newton_zone() in sdc_newton.cuh (Newton
// with pseudo-transient continuation, dense LU with partial pivoting, ties to
// the lowest row).  The zone's matrix and state vectors live in shared memory;
// the work is split across the L lanes: reactions j = lane (mod L) for the
// rate constants and transcendentals, rows i = lane (mod L) for the residual,
// the matrix build and the LU row updates, columns for row exchanges.  Pivot
// search, norms, convergence and admissibility tests and the triangular-solve
// dot products reduce across the group with warp shuffles.
#pragma once
#include "sdc_dev.cuh"

namespace sdcd {

template <int NS, typename MT>
struct GroupLayout {
    static constexpr int N = NS + 1;
    static constexpr int NR = NS - 1;
    // doubles per zone (the matrix rounded up to doubles)
    static constexpr int M_D = (N * N * (int)sizeof(MT) + 7) / 8;
    static constexpr int O_M = 0;
    static constexpr int O_W = O_M + M_D;      // current state w
    static constexpr int O_TR = O_W + N;       // trial state
    static constexpr int O_D = O_TR + N;       // Newton step
    static constexpr int O_G = O_D + N;        // residual at w
    static constexpr int O_GT = O_G + N;       // residual at the trial
    static constexpr int O_K = O_GT + N;       // k_j, dk_j at w
    static constexpr int O_DK = O_K + NR;
    static constexpr int O_KT = O_DK + NR;     // at the trial
    static constexpr int O_DKT = O_KT + NR;
    static constexpr int O_Y = O_DKT + NR;     // Y_i at w, at the trial
    static constexpr int O_YT = O_Y + NS;
    static constexpr int O_R = O_YT + NS;      // reaction rates r_j (scratch)
    static constexpr int O_DR = O_R + NR;      // dr_j/dw_E, dr_j/dw_X0, dr_j/dw_Xj (scratch)
    static constexpr int O_IP = O_DR + 3 * NR; // reciprocal pivots (as MT)
    // the right-hand side / solution of the linear solve as MT: the FP64 slot
    // O_D itself for double, a slot of its own for float (so that the whole
    // solve stays in float: one conversion in, one out)
    static constexpr int V_D = (N * (int)sizeof(MT) + 7) / 8;
    static constexpr int O_DM = sizeof(MT) == 8 ? O_D : O_IP + N;
    static constexpr int RAW = sizeof(MT) == 8 ? O_IP + N : O_DM + V_D;
    static constexpr int STRIDE = RAW | 1;     // odd stride in doubles spreads the banks
};

template <int L>
__device__ __forceinline__ double group_sum(unsigned mask, double v) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

template <int L, typename T>
__device__ __forceinline__ T group_sum_t(unsigned mask, T v) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// |x| as an unsigned integer that orders like |x| (mag2 of sdc_fastmath.cuh)
template <typename MT>
struct AbsBits;
template <>
struct AbsBits<double> {
    using type = unsigned long long;
};
template <>
struct AbsBits<float> {
    using type = unsigned int;
};

template <int L>
__device__ __forceinline__ bool group_all(unsigned mask, bool p) {
    int v = p ? 1 : 0;
#pragma unroll
    for (int o = 1; o < L; o <<= 1) v &= __shfl_xor_sync(mask, v, o);
    return v != 0;
}

// Rate constants, rates and reactive sources of the alpha chain at state w
// (read from zs + O_w), written to the given slots; the residual components of
// this lane's rows to zs + O_g; returns the group's scaled residual norm^2 or
// +inf when T is not positive and finite.
template <int NS, typename MT, int L>
__device__ __forceinline__ double group_eval(const NetParams& P, unsigned mask, int lane, double* zs, int O_w,
                                             int O_k, int O_dk, int O_y, int O_g, double rho, double inv_rho,
                                             double ke, const double* ym, const double* rw_rows, double dtm,
                                             double sE_inv) {
    using Lay = GroupLayout<NS, MT>;
    constexpr int N = Lay::N, NR = Lay::NR;
    constexpr int RL = (N + L - 1) / L;
    const double T = P.gm1 * (zs[O_w] - ke) * inv_rho;
    if (!(T > 0.0 && T < INFINITY)) return INFINITY;
    // Y: species i = lane (mod L)
    for (int i = lane; i < NS; i += L) zs[O_y + i] = zs[O_w + 1 + i] * ym[i];
    // rate constants of this lane's reactions
    const double l2T = log2_tab(T), iT = rcp_nr(T);
    for (int j = lane; j < NR; j += L) {
        const double rp = ipow_small(rho, P.order[j] - 1);
        const double kk = P.a[j] * rp * exp2_tab(P.nu[j] * l2T);
        zs[O_k + j] = kk;
        zs[O_dk + j] = P.nu[j] * kk * iT;
    }
    __syncwarp(mask);
    // rates and the two dense source rows (partial sums over this lane's reactions)
    double sE = 0.0, s0 = 0.0;
    const double y0 = zs[O_y + 0];
    for (int j = lane; j < NR; j += L) {
        const double r = (j == 0) ? zs[O_k + 0] * (y0 * y0 * y0) : zs[O_k + j] * (zs[O_y + j] * y0);
        zs[Lay::O_R + j] = r;
        sE += P.Q[j] * r;
        s0 -= (j == 0 ? 3.0 : 1.0) * r;
    }
    sE = group_sum<L>(mask, sE);
    s0 = group_sum<L>(mask, s0);
    __syncwarp(mask);
    double phi = 0.0;
#pragma unroll
    for (int t = 0; t < RL; t++) {
        const int row = lane + L * t;
        if (row >= N) break;
        double R;
        if (row == 0) {
            R = rho * sE;
        } else if (row == 1) {
            R = rho * P.mass[0] * s0;
        } else {
            const int i = row - 1;  // species i >= 1: made by reaction i-1, used by reaction i
            double S = zs[Lay::O_R + i - 1];
            if (i < NR) S -= zs[Lay::O_R + i];
            R = rho * P.mass[i] * S;
        }
        const double G = zs[O_w + row] - dtm * R - rw_rows[t];
        zs[O_g + row] = G;
        const double gs = row == 0 ? G * sE_inv : G * inv_rho;
        phi += gs * gs;
    }
    phi = group_sum<L>(mask, phi);
    return phi < INFINITY ? phi : INFINITY;
}

template <int NS, typename MT, int L>
__device__ __forceinline__ int newton_zone_group(const NetParams& P, const NewtonCfg& cfg, unsigned mask, int lane,
                                                 double* zs, double rho, double m2, const double* rw_rows,
                                                 double dtm, int& iters) {
    using Lay = GroupLayout<NS, MT>;
    constexpr int N = Lay::N, NR = Lay::NR;
    constexpr int RL = (N + L - 1) / L;
    MT* M = reinterpret_cast<MT*>(zs + Lay::O_M);
    MT* dm = reinterpret_cast<MT*>(zs + Lay::O_DM);   // right-hand side, then the Newton step
    MT* ipm = reinterpret_cast<MT*>(zs + Lay::O_IP);  // reciprocal pivots
    using IT = typename AbsBits<MT>::type;
    const double inv_rho = rcp_nr(rho);
    const double ke = 0.5 * m2 * inv_rho;
    double ym[NS];
#pragma unroll
    for (int i = 0; i < NS; i++) ym[i] = inv_rho * P.inv_mass[i];
    const double rwE = __shfl_sync(mask, rw_rows[0], (threadIdx.x & 31) & ~(L - 1));  // row 0 lives on lane 0
    const double sE_inv = rcp_nr(fabs(rwE));

    // a start without a positive temperature is replaced by rhs (rows of this lane)
    {
        const double Tg = P.gm1 * (zs[Lay::O_W] - ke) * inv_rho;
        const bool bad = !(Tg > 0.0 && Tg < INFINITY);
        __syncwarp(mask);
        if (bad) {
#pragma unroll
            for (int t = 0; t < RL; t++) {
                const int row = lane + L * t;
                if (row < N) zs[Lay::O_W + row] = rw_rows[t];
            }
        }
        __syncwarp(mask);
    }
    // admissibility floor on rho X_i for this lane's species rows; it applies
    // when the rhs is physical (every X_i >= -0.01)
    bool physical = true;
#pragma unroll
    for (int t = 0; t < RL; t++) {
        const int row = lane + L * t;
        if (row >= 1 && row < N) physical = physical && (rw_rows[t] * inv_rho >= -XMARGIN);
    }
    physical = group_all<L>(mask, physical);
    double lower[RL];
#pragma unroll
    for (int t = 0; t < RL; t++) {
        const int row = lane + L * t;
        lower[t] = -INFINITY;
        if (physical && row >= 1 && row < N) {
            const double x = rw_rows[t] * inv_rho, xg = zs[Lay::O_W + row] * inv_rho;
            double lo = x < 0.0 ? x : 0.0;
            lo = xg < lo ? xg : lo;
            lower[t] = (lo - XMARGIN) * rho;
        }
    }
    double phi = group_eval<NS, MT, L>(P, mask, lane, zs, Lay::O_W, Lay::O_K, Lay::O_DK, Lay::O_Y, Lay::O_G, rho,
                                       inv_rho, ke, ym, rw_rows, dtm, sE_inv);
    const bool have_k = phi < INFINITY;
    int status = ZONE_MAXIT;
    iters = 0;
    if (!have_k) {
        status = ZONE_NONPHYSICAL;
    } else {
        bool newton = true;
        double h = PTC_H0;
        int it;
        for (it = 1; it <= cfg.maxit; it++) {
            const double c = newton ? 1.0 : 1.0 + rcp_nr(h);
            // ---- derivative terms of this lane's reactions at w
            const double dTdE = P.gm1 * inv_rho;
            const double y0 = zs[Lay::O_Y + 0];
            for (int j = lane; j < NR; j += L) {
                double drE, drX0, drXj = 0.0;
                if (j == 0) {
                    drE = zs[Lay::O_DK + 0] * (y0 * y0 * y0) * dTdE;
                    drX0 = zs[Lay::O_K + 0] * (3.0 * y0 * y0) * ym[0];
                } else {
                    const double yj = zs[Lay::O_Y + j];
                    drE = zs[Lay::O_DK + j] * (yj * y0) * dTdE;
                    drXj = zs[Lay::O_K + j] * y0 * ym[j];
                    drX0 = zs[Lay::O_K + j] * yj * ym[0];
                }
                zs[Lay::O_DR + 3 * j + 0] = drE;
                zs[Lay::O_DR + 3 * j + 1] = drX0;
                zs[Lay::O_DR + 3 * j + 2] = drXj;
            }
            __syncwarp(mask);
            // ---- matrix rows of this lane: M = c I - dtm dR/dw; d = G
            const double s = dtm * rho;
#pragma unroll
            for (int t = 0; t < RL; t++) {
                const int row = lane + L * t;
                if (row >= N) break;
                MT* Mr = M + row * N;
#pragma unroll
                for (int q = 0; q < N; q++) Mr[q] = (q == row) ? (MT)c : (MT)0;
                if (row == 0) {
                    for (int j = 0; j < NR; j++) {
                        const double qj = s * P.Q[j];
                        Mr[0] -= (MT)(qj * zs[Lay::O_DR + 3 * j]);
                        Mr[1] -= (MT)(qj * zs[Lay::O_DR + 3 * j + 1]);
                        if (j > 0) Mr[1 + j] -= (MT)(qj * zs[Lay::O_DR + 3 * j + 2]);
                    }
                } else if (row == 1) {
                    for (int j = 0; j < NR; j++) {
                        const double a0 = s * P.mass[0] * (j == 0 ? -3.0 : -1.0);
                        Mr[0] -= (MT)(a0 * zs[Lay::O_DR + 3 * j]);
                        Mr[1] -= (MT)(a0 * zs[Lay::O_DR + 3 * j + 1]);
                        if (j > 0) Mr[1 + j] -= (MT)(a0 * zs[Lay::O_DR + 3 * j + 2]);
                    }
                } else {
                    const int i = row - 1;
                    // made by reaction i-1 (+1), used by reaction i (-1)
                    {
                        const int j = i - 1;
                        const double ap = s * P.mass[i];
                        Mr[0] -= (MT)(ap * zs[Lay::O_DR + 3 * j]);
                        Mr[1] -= (MT)(ap * zs[Lay::O_DR + 3 * j + 1]);
                        if (j > 0) Mr[1 + j] -= (MT)(ap * zs[Lay::O_DR + 3 * j + 2]);
                    }
                    if (i < NR) {
                        const int j = i;
                        const double am = -s * P.mass[i];
                        Mr[0] -= (MT)(am * zs[Lay::O_DR + 3 * j]);
                        Mr[1] -= (MT)(am * zs[Lay::O_DR + 3 * j + 1]);
                        Mr[1 + j] -= (MT)(am * zs[Lay::O_DR + 3 * j + 2]);
                    }
                }
                dm[row] = (MT)zs[Lay::O_G + row];
            }
            __syncwarp(mask);
            // ---- LU with partial pivoting, rows exchanged column-wise across the lanes
            bool singular = false;
            for (int k = 0; k < N; k++) {
                // pivot: largest |M[i][k]|, i >= k, ties to the lowest row (|x|
                // compared as bit patterns on the integer pipe: they order like the values)
                IT best = 0;
                int piv = N;
                for (int i = k + lane; i < N; i += L) {
                    const IT v = mag2(M[i * N + k]);
                    if (v > best || piv == N) { best = v; piv = i; }
                }
#pragma unroll
                for (int o = 1; o < L; o <<= 1) {
                    const IT ob = __shfl_xor_sync(mask, best, o);
                    const int op = __shfl_xor_sync(mask, piv, o);
                    if (ob > best || (ob == best && op < piv)) { best = ob; piv = op; }
                }
                if (!(best > 0)) { singular = true; break; }
                if (piv != k) {
                    for (int q = k + lane; q < N; q += L) {
                        const MT a = M[k * N + q];
                        M[k * N + q] = M[piv * N + q];
                        M[piv * N + q] = a;
                    }
                    if (lane == 0) {
                        const MT a = dm[k];
                        dm[k] = dm[piv];
                        dm[piv] = a;
                    }
                }
                __syncwarp(mask);
                const MT pv = M[k * N + k];
                const MT ip = (sizeof(MT) == 8) ? (MT)rcp_nr((double)pv) : (MT)1 / pv;
                if (lane == 0) ipm[k] = ip;
                const MT dk_ = dm[k];
                for (int i = k + 1 + lane; i < N; i += L) {
                    const MT l = M[i * N + k] * ip;
                    M[i * N + k] = l;
                    for (int q = k + 1; q < N; q++) M[i * N + q] -= l * M[k * N + q];
                    dm[i] -= l * dk_;
                }
                __syncwarp(mask);
            }
            if (singular) { status = ZONE_SINGULAR; break; }
            // ---- back substitution (dot products split across the lanes)
            for (int i = N - 1; i >= 0; i--) {
                MT part = 0;
                for (int q = i + 1 + lane; q < N; q += L) part += M[i * N + q] * dm[q];
                part = group_sum_t<L, MT>(mask, part);
                if (lane == 0) dm[i] = (dm[i] - part) * ipm[i];
                __syncwarp(mask);
            }
            if (sizeof(MT) != 8) {
                for (int r = lane; r < N; r += L) zs[Lay::O_D + r] = (double)dm[r];
                __syncwarp(mask);
            }
            // ---- trial state, admissibility, residual at the trial
            bool ok = true;
#pragma unroll
            for (int t = 0; t < RL; t++) {
                const int row = lane + L * t;
                if (row >= N) break;
                const double tr = zs[Lay::O_W + row] - zs[Lay::O_D + row];
                zs[Lay::O_TR + row] = tr;
                if (row >= 1) ok = ok && (tr >= lower[t]);
            }
            ok = group_all<L>(mask, ok);
            __syncwarp(mask);
            double phit = INFINITY;
            if (ok)
                phit = group_eval<NS, MT, L>(P, mask, lane, zs, Lay::O_TR, Lay::O_KT, Lay::O_DKT, Lay::O_YT, Lay::O_GT,
                                             rho, inv_rho, ke, ym, rw_rows, dtm, sE_inv);
            ok = ok && phit < INFINITY;
            // an admissible Newton step that meets the stop test converges even
            // if the residual grew by round-off at the root
            bool small = false;
            if (newton && ok) {
                const double trE = zs[Lay::O_TR + 0];
                small = true;
#pragma unroll
                for (int t = 0; t < RL; t++) {
                    const int row = lane + L * t;
                    if (row >= N) break;
                    const double dd = fabs(zs[Lay::O_D + row]);
                    small = small && (row == 0 ? dd <= cfg.rtol * fabs(trE) : dd <= cfg.rtol * rho);
                }
                small = group_all<L>(mask, small);
            }
            if (newton && !small && (!ok || phit > phi)) {
                newton = false;
                h = PTC_H0;
                __syncwarp(mask);
                continue;
            }
            if (!ok) {
                h /= PTC_SHRINK;
                __syncwarp(mask);
                if (h < PTC_HMIN) { status = ZONE_NONPHYSICAL; break; }
                continue;
            }
            // ---- take the trial
            for (int r = lane; r < N; r += L) {
                zs[Lay::O_W + r] = zs[Lay::O_TR + r];
                zs[Lay::O_G + r] = zs[Lay::O_GT + r];
            }
            for (int j = lane; j < NR; j += L) {
                zs[Lay::O_K + j] = zs[Lay::O_KT + j];
                zs[Lay::O_DK + j] = zs[Lay::O_DKT + j];
            }
            for (int i = lane; i < NS; i += L) zs[Lay::O_Y + i] = zs[Lay::O_YT + i];
            phi = phit;
            __syncwarp(mask);
            if (newton) {
                if (small) { status = ZONE_OK; break; }
            } else {
                h *= PTC_GROW;
                if (h >= PTC_HNEWTON) newton = true;
            }
        }
        iters = it > cfg.maxit ? cfg.maxit : it;
    }
    __syncwarp(mask);
    // reactive source at the final state: rows of this lane into zs + O_G (as R, not G)
    if (!have_k) {
        // fall back to a fresh evaluation (T not positive: the rates are not finite)
        const double T = P.gm1 * (zs[Lay::O_W] - ke) * inv_rho;
        const double l2T = log2_tab(T);
        for (int j = lane; j < NR; j += L) {
            zs[Lay::O_K + j] = P.a[j] * ipow_small(rho, P.order[j] - 1) * exp2_tab(P.nu[j] * l2T);
        }
        for (int i = lane; i < NS; i += L) zs[Lay::O_Y + i] = zs[Lay::O_W + 1 + i] * ym[i];
        __syncwarp(mask);
    }
    double sE = 0.0, s0 = 0.0;
    const double y0 = zs[Lay::O_Y + 0];
    for (int j = lane; j < NR; j += L) {
        const double r = (j == 0) ? zs[Lay::O_K + 0] * (y0 * y0 * y0) : zs[Lay::O_K + j] * (zs[Lay::O_Y + j] * y0);
        zs[Lay::O_R + j] = r;
        sE += P.Q[j] * r;
        s0 -= (j == 0 ? 3.0 : 1.0) * r;
    }
    sE = group_sum<L>(mask, sE);
    s0 = group_sum<L>(mask, s0);
    __syncwarp(mask);
#pragma unroll
    for (int t = 0; t < RL; t++) {
        const int row = lane + L * t;
        if (row >= N) break;
        double R;
        if (row == 0) R = rho * sE;
        else if (row == 1) R = rho * P.mass[0] * s0;
        else {
            const int i = row - 1;
            double S = zs[Lay::O_R + i - 1];
            if (i < NR) S -= zs[Lay::O_R + i];
            R = rho * P.mass[i] * S;
        }
        zs[Lay::O_G + row] = R;
    }
    __syncwarp(mask);
    return status;
}

}  // namespace sdcd
