// sdc_adjoint.cu -- kernels of the adjoint of one SDC step (paper section 2,
// Eq. sdc:general): the advective-term VJP (per face, forward mode, then a
// deterministic per-zone gather), the VJP of the reactive source and of the
// implicit reaction update (implicit-function theorem: a transposed solve with
// the Jacobian at the converged root), the adjoint of the right-hand side, and
// a fixed-order reduction of the rate-prefactor gradient.
#include "sdc_adjoint.cuh"
#include "sdc_adjoint_launch.h"

namespace sdcd {

constexpr int ADJ_BLOCK = 128;

__device__ __forceinline__ int box_of(const BoxDev* boxes, int nbox, long long z) {
    int lo = 0, hi = nbox - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (boxes[mid].off <= z) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// global index of the zone shifted by o along dir inside its (periodic) box
// (32-bit arithmetic inside the box: a box holds fewer than 2^31 zones, and
// 64-bit division would run on the narrow FP64 pipe)
__device__ __forceinline__ long long shifted(const BoxDev& b, long long z, int dir, int o) {
    const int l = (int)(z - b.off);
    int c[3];
    c[0] = l % b.n[0];
    c[1] = (l / b.n[0]) % b.n[1];
    c[2] = l / (b.n[0] * b.n[1]);
    c[dir] = ((c[dir] + o) % b.n[dir] + b.n[dir]) % b.n[dir];
    return b.off + (long long)(c[0] + b.n[0] * (c[1] + b.n[1] * c[2]));
}

// G[dir][4*NV][z] (field-major, so that the writes here and the reads of the
// gather are coalesced): transposed Jacobian of the flux through the face
// between z and z+1 (along dir) times that face's adjoint, for the inputs of
// zones z-1, z, z+1, z+2 (slot o*NV + f).
template <int DIM, int NS>
__global__ void __launch_bounds__(ADJ_BLOCK)
stencil_vjp_kernel(double gamma, int limiter, long long N, const BoxDev* __restrict__ boxes, int nbox,
                   const double* __restrict__ U, const double* __restrict__ Abar, double* __restrict__ G) {
    constexpr int NV = 2 + DIM + NS;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * DIM) return;
    const int dir = (int)(t / N);
    const long long z = t - (long long)dir * N;
    const BoxDev b = boxes[box_of(boxes, nbox, z)];
    long long zz[4];
#pragma unroll
    for (int o = 0; o < 4; o++) zz[o] = shifted(b, z, dir, o - 1);
    // face adjoint: A_l -= F idx, A_{l+1} += F idx
    double Fbar[NV];
#pragma unroll
    for (int f = 0; f < NV; f++) Fbar[f] = (Abar[f * N + zz[2]] - Abar[f * N + zz[1]]) * b.idx[dir];
    Dual Uz[4][NV];
#pragma unroll
    for (int o = 0; o < 4; o++)
#pragma unroll
        for (int f = 0; f < NV; f++) Uz[o][f] = Dual(U[f * N + zz[o]], 0.0);
    double* out = G + (long long)dir * N * (4 * NV) + z;
    for (int j = 0; j < 4 * NV; j++) {
        const int o = j / NV, f = j % NV;
        Uz[o][f].d = 1.0;
        Dual F[NV];
        face_flux_dual<DIM, NS>(gamma, limiter, dir, Uz, F);
        Uz[o][f].d = 0.0;
        double c = 0.0;
#pragma unroll
        for (int q = 0; q < NV; q++) c += Fbar[q] * F[q].d;
        out[(long long)j * N] = c;
    }
}

// Same product as stencil_vjp_kernel, by a reverse sweep through the face flux.
template <int DIM, int NS>
__global__ void __launch_bounds__(ADJ_BLOCK)
stencil_vjp_rev_kernel(double gamma, int limiter, long long N, const BoxDev* __restrict__ boxes, int nbox,
                       const double* __restrict__ U, const double* __restrict__ Abar, double* __restrict__ G) {
    constexpr int NV = 2 + DIM + NS;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * DIM) return;
    const int dir = (int)(t / N);
    const long long z = t - (long long)dir * N;
    const BoxDev b = boxes[box_of(boxes, nbox, z)];
    long long zz[4];
#pragma unroll
    for (int o = 0; o < 4; o++) zz[o] = shifted(b, z, dir, o - 1);
    double Fbar[NV];
#pragma unroll
    for (int f = 0; f < NV; f++) Fbar[f] = (Abar[f * N + zz[2]] - Abar[f * N + zz[1]]) * b.idx[dir];
    double Uz[4][NV], Ub[4][NV];
#pragma unroll
    for (int o = 0; o < 4; o++)
#pragma unroll
        for (int f = 0; f < NV; f++) {
            Uz[o][f] = U[f * N + zz[o]];
            Ub[o][f] = 0.0;
        }
    face_flux_vjp<DIM, NS>(gamma, limiter, dir, Uz, Fbar, Ub);
    double* out = G + (long long)dir * N * (4 * NV) + z;
#pragma unroll
    for (int o = 0; o < 4; o++)
#pragma unroll
        for (int f = 0; f < NV; f++) out[(long long)(o * NV + f) * N] = Ub[o][f];
}

// Ubar_z += sum over directions and over the four faces whose stencil holds z
template <int DIM, int NS>
__global__ void __launch_bounds__(ADJ_BLOCK)
stencil_vjp_gather(long long N, const BoxDev* __restrict__ boxes, int nbox, const double* __restrict__ G,
                   double* __restrict__ Ubar) {
    constexpr int NV = 2 + DIM + NS;
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const BoxDev b = boxes[box_of(boxes, nbox, z)];
    double acc[NV];
#pragma unroll
    for (int f = 0; f < NV; f++) acc[f] = 0.0;
    for (int dir = 0; dir < DIM; dir++)
#pragma unroll
        for (int o = 0; o < 4; o++) {
            // z is input slot o of the face whose left zone is z + 1 - o
            const long long l = shifted(b, z, dir, 1 - o);
            const double* g = G + (long long)dir * N * (4 * NV) + (long long)(o * NV) * N + l;
#pragma unroll
            for (int f = 0; f < NV; f++) acc[f] += g[(long long)f * N];
        }
#pragma unroll
    for (int f = 0; f < NV; f++) Ubar[f * N + z] += acc[f];
}

// dR/dw (n x n, row = reactive field, col = unknown), dR/da_j (n x nr) and R
// at the state (rho, mom, w) of an alpha chain or a generic network.
template <int NS, int TOPO>
__device__ __forceinline__ void reaction_derivs(const NetParams& P, double rho, double m2, const double* w,
                                                double (*dR)[NS + 1], double (*dRa)[NS - 1]) {
    constexpr int N = NS + 1;
    constexpr int NR = NS - 1;
    const double inv_rho = rcp_nr(rho);
    const double T = P.gm1 * (w[0] - 0.5 * m2 * inv_rho) * inv_rho;
    double k[NR], dk[NR], Y[NS];
    rate_consts<NR>(P, rho, T, k, dk);
    double ym[NS];
#pragma unroll
    for (int i = 0; i < NS; i++) ym[i] = inv_rho * P.inv_mass[i];
#pragma unroll
    for (int i = 0; i < NS; i++) Y[i] = w[1 + i] * ym[i];
    // M = 0 I - 1 * dR/dw = -dR/dw  (build_matrix with c = 0, dtm = 1)
    double M[N][N];
    build_matrix<NS, TOPO, double>(P, rho, inv_rho, ym, k, dk, Y, 0.0, 1.0, M);
#pragma unroll
    for (int r = 0; r < N; r++)
#pragma unroll
        for (int c = 0; c < N; c++) dR[r][c] = -M[r][c];
    // dR/da_j = (R with only reaction j, at a_j = 1): R_r = rho C_rj r_j, r_j linear in a_j
#pragma unroll
    for (int j = 0; j < NR; j++) {
        double kj[NR];
#pragma unroll
        for (int q = 0; q < NR; q++) kj[q] = 0.0;
        kj[j] = (P.a[j] != 0.0) ? k[j] * rcp_nr(P.a[j]) : ipow_small(rho, P.order[j] - 1) *
                                                   (P.law == LAW_POWER ? exp2_tab(P.nu[j] * log2_tab(T)) : exp(-P.nu[j] / T));
        double Rj[N];
        sources<NS, TOPO>(P, rho, kj, Y, Rj);
#pragma unroll
        for (int r = 0; r < N; r++) dRa[r][j] = Rj[r];
    }
}

// ---- the alpha chain: the same VJP without dense matrices
// With q_j = rho r_j = kappa_j P_j (kappa_j = amp_j f_j(T), P_0 = w_0^3,
// P_j = w_0 w_j) the sources are R = sum_j sigma_j q_j, sigma_j reaction j's
// column (Q_j in the energy row, mass_i s_ij in species row i), so for any v
//   (dR/dw)^T v = sum_j (sigma_j . v) dq_j/dw,   (dR/da_j)^T v = (sigma_j . v) q_j / a_j,
// where dq_j/dw has at most three nonzero entries (rho E through T, X_0, X_j).
// The transposed solve (I - dt_m dR/dw)^T lambda = b uses the bordered chain
// elimination of the forward Newton step: M^T in reversed chain order
// (X_{n-1} .. X_1) is again lower bidiagonal in the chain, bordered by the
// energy and alpha rows and columns.
template <int NS>
struct ChainDerivs {
    static constexpr int NR = NS - 1;
    double q[NR];    // q_j = kappa_j P_j
    double dE[NR];   // dq_j / d(rho E) = q_j nu_j f (gamma-1) / rho
    double d0[NR];   // dq_j / dw_0
    double dj[NR];   // dq_j / dw_j (j >= 1)
    double fa[NR];   // q_j / a_j = f_j(T) P_j / prod of the reactant masses
};

// sigma_j . v (v in w order: rho E, rho X_0, ..)
template <int NS>
__device__ __forceinline__ double chain_sigma_dot(const NetParams& P, int j, const double* v) {
    double s = fma(P.Q[j], v[0], P.rs[j][0] * v[1]);
    if (j >= 1) s = fma(P.rs[j][1], v[1 + j], s);
    return fma(P.rs[j][2], v[2 + j], s);
}

// out = (dR/dw)^T v, and sv[j] = sigma_j . v
template <int NS>
__device__ __forceinline__ void chain_dRT(const NetParams& P, const ChainDerivs<NS>& D, const double* v, double* out,
                                          double* sv) {
    constexpr int N = NS + 1;
    constexpr int NR = NS - 1;
#pragma unroll
    for (int r = 0; r < N; r++) out[r] = 0.0;
#pragma unroll
    for (int j = 0; j < NR; j++) {
        const double sj = chain_sigma_dot<NS>(P, j, v);
        sv[j] = sj;
        out[0] = fma(sj, D.dE[j], out[0]);
        out[1] = fma(sj, D.d0[j], out[1]);
        if (j >= 1) out[1 + j] = fma(sj, D.dj[j], out[1 + j]);
    }
}

// Solve (I - dtm dR/dw)^T lambda = b in place (b, lambda in w order).
template <int NS>
__device__ __forceinline__ bool chain_solve_transposed(const NetParams& P, const double* kap, double dfac_rho,
                                                       const double* ws, double dtm, double* b) {
    constexpr int NC = NS - 1;
    ChainSys<NS, double> A, At;
    build_chain<NS, double>(P, kap, dfac_rho, ws, 1.0, dtm, A);
    // M^T with the chain reversed: chain position k of At is species X_{NC-k}
#pragma unroll
    for (int k = 0; k < NC; k++) {
        const int o = NC - 1 - k;
        At.bd[k] = A.bd[o];
        At.bs[k] = k >= 1 ? A.bs[o + 1] : 0.0;  // M^T[X_{o+1}][X_{o+2}] = M[X_{o+2}][X_{o+1}]
        At.uE[k] = A.vE[o];
        At.uA[k] = A.vA[o];
        At.vE[k] = A.uE[o];
        At.vA[k] = A.uA[o];
    }
    At.dEE = A.dEE; At.dEA = A.dAE; At.dAE = A.dEA; At.dAA = A.dAA;
    double x[NS + 1];
    x[0] = b[0];
    x[1] = b[1];
#pragma unroll
    for (int k = 0; k < NC; k++) x[2 + k] = b[2 + NC - 1 - k];
    const bool ok = chain_solve<NS, double>(At, x);
    b[0] = x[0];
    b[1] = x[1];
#pragma unroll
    for (int k = 0; k < NC; k++) b[2 + NC - 1 - k] = x[2 + k];
    return ok;
}

// Reactive-source VJP at the state U (with Rbar) and, when dtm > 0, the VJP of
// the implicit update whose root is U: rhsbar = d rhs.  abar_zone[j*N + z] +=.
template <int NS, int TOPO>
__global__ void __launch_bounds__(ADJ_BLOCK)
reaction_vjp_kernel(NetParams P, long long N, int dim, const double* __restrict__ U, const double* __restrict__ Rbar,
                    double* __restrict__ Ubar, double dtm, double* __restrict__ rhsbar,
                    double* __restrict__ abar_zone) {
    constexpr int NW = NS + 1;
    constexpr int NR = NS - 1;
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const double rho = U[z];
    double mom[3] = {0.0, 0.0, 0.0}, m2 = 0.0;
    for (int d = 0; d < dim; d++) {
        mom[d] = U[(1 + d) * N + z];
        m2 += mom[d] * mom[d];
    }
    double w[NW];
#pragma unroll
    for (int r = 0; r < NW; r++) w[r] = U[(1 + dim + r) * N + z];
    double dR[NW][NW], dRa[NW][NR];
    reaction_derivs<NS, TOPO>(P, rho, m2, w, dR, dRa);
    const double irho = rcp_nr(rho);
    const double cE_rho = -w[0] * irho + m2 * (irho * irho);  // dT/d(rho) / dT/d(rho E)
    double ub_rho = Ubar[z], ub_m[3] = {0.0, 0.0, 0.0}, ub_w[NW];
    for (int d = 0; d < dim; d++) ub_m[d] = Ubar[(1 + d) * N + z];
#pragma unroll
    for (int r = 0; r < NW; r++) ub_w[r] = Ubar[(1 + dim + r) * N + z];
    double ga[NR];
#pragma unroll
    for (int j = 0; j < NR; j++) ga[j] = 0.0;
    if (Rbar) {
        double rb[NW];
#pragma unroll
        for (int r = 0; r < NW; r++) rb[r] = Rbar[r * N + z];
#pragma unroll
        for (int c = 0; c < NW; c++) {
            double s = 0.0;
#pragma unroll
            for (int r = 0; r < NW; r++) s += dR[r][c] * rb[r];
            ub_w[c] += s;
        }
        double DE = 0.0;
#pragma unroll
        for (int r = 0; r < NW; r++) DE += rb[r] * dR[r][0];
        ub_rho += DE * cE_rho;
        for (int d = 0; d < dim; d++) ub_m[d] -= DE * mom[d] * irho;
#pragma unroll
        for (int j = 0; j < NR; j++) {
            double s = 0.0;
#pragma unroll
            for (int r = 0; r < NW; r++) s += rb[r] * dRa[r][j];
            ga[j] += s;
        }
    }
    if (dtm > 0.0) {
        // J^T lambda = ub_w, J = I - dtm dR/dw
        double JT[NW][NW];
#pragma unroll
        for (int r = 0; r < NW; r++)
#pragma unroll
            for (int c = 0; c < NW; c++) JT[c][r] = (r == c ? 1.0 : 0.0) - dtm * dR[r][c];
        double lam[NW];
#pragma unroll
        for (int r = 0; r < NW; r++) lam[r] = ub_w[r];
        if (!lu_solve<NW, double, double>(JT, lam)) {
            // singular Jacobian at the root: the update is not differentiable here
#pragma unroll
            for (int r = 0; r < NW; r++) lam[r] = 0.0;
        }
        double DE = 0.0;
#pragma unroll
        for (int r = 0; r < NW; r++) DE += lam[r] * dR[r][0];
        rhsbar[z] = ub_rho + dtm * DE * cE_rho;
        for (int d = 0; d < dim; d++) rhsbar[(1 + d) * N + z] = ub_m[d] - dtm * DE * mom[d] * irho;
#pragma unroll
        for (int r = 0; r < NW; r++) rhsbar[(1 + dim + r) * N + z] = lam[r];
#pragma unroll
        for (int j = 0; j < NR; j++) {
            double s = 0.0;
#pragma unroll
            for (int r = 0; r < NW; r++) s += lam[r] * dRa[r][j];
            ga[j] += dtm * s;
        }
    } else {
        Ubar[z] = ub_rho;
        for (int d = 0; d < dim; d++) Ubar[(1 + d) * N + z] = ub_m[d];
#pragma unroll
        for (int r = 0; r < NW; r++) Ubar[(1 + dim + r) * N + z] = ub_w[r];
    }
#pragma unroll
    for (int j = 0; j < NR; j++) abar_zone[j * N + z] += ga[j];
}

// reaction_vjp_kernel for the alpha chain (any length, 13 species included),
// from the per-reaction derivatives of ChainDerivs: O(n) work and registers
// per zone instead of the dense n x n Jacobian and n x (n-1) rate derivatives.
template <int NS>
__global__ void __launch_bounds__(ADJ_BLOCK)
reaction_vjp_chain_kernel(NetParams P, long long N, int dim, const double* __restrict__ U,
                          const double* __restrict__ Rbar, double* __restrict__ Ubar, double dtm,
                          double* __restrict__ rhsbar, double* __restrict__ abar_zone) {
    constexpr int NW = NS + 1;
    constexpr int NR = NS - 1;
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const double rho = U[z];
    double mom[3] = {0.0, 0.0, 0.0}, m2 = 0.0;
    for (int d = 0; d < dim; d++) {
        mom[d] = U[(1 + d) * N + z];
        m2 += mom[d] * mom[d];
    }
    double w[NW];
#pragma unroll
    for (int r = 0; r < NW; r++) w[r] = U[(1 + dim + r) * N + z];
    const double irho = rcp_nr(rho);
    const double T = P.gm1 * (w[0] - 0.5 * m2 * irho) * irho;
    // kappa_j = amp_j f_j(T) and f_j(T) alone (unit prefactors), dfac = d ln f_j / dT / nu_j
    double kap[NR], f[NR], dfac;
    {
        double one[NR];
#pragma unroll
        for (int j = 0; j < NR; j++) one[j] = 1.0;
        rate_consts_k<NR>(P, one, T, f, dfac);
#pragma unroll
        for (int j = 0; j < NR; j++) kap[j] = P.amp[j] * f[j];
    }
    ChainDerivs<NS> D;
    const double gE = P.gm1 * dfac * irho;  // dT/d(rho E) times dfac
#pragma unroll
    for (int j = 0; j < NR; j++) {
        const double w0 = w[1], wj = w[1 + j];
        const double Pj = j == 0 ? w0 * w0 * w0 : w0 * wj;
        D.q[j] = kap[j] * Pj;
        D.dE[j] = D.q[j] * P.nu[j] * gE;
        D.d0[j] = j == 0 ? 3.0 * kap[0] * (w0 * w0) : kap[j] * wj;
        D.dj[j] = j == 0 ? 0.0 : kap[j] * w0;
        // the reactant masses' product: 1 / prod mass = amp_j / a_j (a_j may be 0)
        const double mp = j == 0 ? P.mass[0] * P.mass[0] * P.mass[0] : P.mass[j] * P.mass[0];
        D.fa[j] = f[j] * Pj * rcp_nr(mp);
    }
    const double cE_rho = -w[0] * irho + m2 * (irho * irho);  // dT/d(rho) / dT/d(rho E)
    double ub_rho = Ubar[z], ub_m[3] = {0.0, 0.0, 0.0}, ub_w[NW];
    for (int d = 0; d < dim; d++) ub_m[d] = Ubar[(1 + d) * N + z];
#pragma unroll
    for (int r = 0; r < NW; r++) ub_w[r] = Ubar[(1 + dim + r) * N + z];
    double ga[NR];
#pragma unroll
    for (int j = 0; j < NR; j++) ga[j] = 0.0;
    if (Rbar) {
        double rb[NW], t[NW], sv[NR];
#pragma unroll
        for (int r = 0; r < NW; r++) rb[r] = Rbar[r * N + z];
        chain_dRT<NS>(P, D, rb, t, sv);
#pragma unroll
        for (int c = 0; c < NW; c++) ub_w[c] += t[c];
        const double DE = t[0];
        ub_rho += DE * cE_rho;
        for (int d = 0; d < dim; d++) ub_m[d] -= DE * mom[d] * irho;
#pragma unroll
        for (int j = 0; j < NR; j++) ga[j] += sv[j] * D.fa[j];
    }
    if (dtm > 0.0) {
        double lam[NW];
#pragma unroll
        for (int r = 0; r < NW; r++) lam[r] = ub_w[r];
        if (!chain_solve_transposed<NS>(P, kap, dfac * irho, w + 1, dtm, lam)) {
            // singular Jacobian at the root: the update is not differentiable here
#pragma unroll
            for (int r = 0; r < NW; r++) lam[r] = 0.0;
        }
        double t[NW], sv[NR];
        chain_dRT<NS>(P, D, lam, t, sv);
        const double DE = t[0];
        rhsbar[z] = ub_rho + dtm * DE * cE_rho;
        for (int d = 0; d < dim; d++) rhsbar[(1 + d) * N + z] = ub_m[d] - dtm * DE * mom[d] * irho;
#pragma unroll
        for (int r = 0; r < NW; r++) rhsbar[(1 + dim + r) * N + z] = lam[r];
#pragma unroll
        for (int j = 0; j < NR; j++) ga[j] += dtm * (sv[j] * D.fa[j]);
    } else {
        Ubar[z] = ub_rho;
        for (int d = 0; d < dim; d++) Ubar[(1 + d) * N + z] = ub_m[d];
#pragma unroll
        for (int r = 0; r < NW; r++) Ubar[(1 + dim + r) * N + z] = ub_w[r];
    }
#pragma unroll
    for (int j = 0; j < NR; j++) abar_zone[j * N + z] += ga[j];
}

// adjoint of rhs_m = U_m + dtm (A_m_new - A_m_old) - dtm R_{m+1}_old + sum_l q_l dt (A_l_old + R_l_old)
__global__ void rhs_adjoint_kernel(RhsAdjArgs a) {
    // one thread per zone, every field (no 64-bit division per element)
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= a.N) return;
    for (int f = 0; f < a.nvar; f++) {
        const long long i = (long long)f * a.N + z;
        const double g = a.rhsbar[i];
        const bool reactive = f >= 1 + a.dim;
        const long long ir = (long long)(f - 1 - a.dim) * a.N + z;
        a.Ubar_m[i] += g;
        if (a.Abar_new_m) {
            a.Abar_new_m[i] += a.dtm * g;
            a.Abar_old[a.m][i] -= a.dtm * g;
        }
        if (reactive) a.Rbar_old[a.m + 1][ir] -= a.dtm * g;
        for (int l = 0; l < a.M; l++) {
            a.Abar_old[l][i] += a.qdt[l] * g;
            if (reactive) a.Rbar_old[l][ir] += a.qdt[l] * g;
        }
    }
}

// g_a[j] += sum_z abar_zone[j*N + z] (fixed order: one block per reaction)
__global__ void reduce_rows_kernel(long long N, const double* __restrict__ x, double* __restrict__ out) {
    __shared__ double s[256];
    const int j = blockIdx.x;
    double acc = 0.0;
    for (long long z = threadIdx.x; z < N; z += blockDim.x) acc += x[(long long)j * N + z];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] += s[0];
}

// ---------------------------------------------------------------- dispatch
#define SDC_ADJ_CASES(X) \
    X(1, 2, TOPO_GENERIC) \
    X(3, 2, TOPO_GENERIC) \
    X(3, 5, TOPO_CHAIN)   \
    X(3, 7, TOPO_CHAIN)   \
    X(3, 13, TOPO_CHAIN)

bool adjoint_supported(int dim, int nspec, int topo) {
#define X(d, ns, tp) \
    if (dim == d && nspec == ns && topo == tp) return true;
    SDC_ADJ_CASES(X)
#undef X
    return false;
}

cudaError_t launch_stencil_vjp(const NetParams& P, int dim, int limiter, long long N, const BoxDev* boxes, int nbox,
                               const double* U, const double* Abar, double* G, double* Ubar, cudaStream_t st,
                               int mode) {
    const unsigned g1 = (unsigned)((N * dim + ADJ_BLOCK - 1) / ADJ_BLOCK);
    const unsigned g2 = (unsigned)((N + ADJ_BLOCK - 1) / ADJ_BLOCK);
#define X(d, ns, tp)                                                                                            \
    if (dim == d && P.nspec == ns && P.topo == tp) {                                                            \
        if (mode == 0)                                                                                          \
            stencil_vjp_rev_kernel<d, ns><<<g1, ADJ_BLOCK, 0, st>>>(P.gamma, limiter, N, boxes, nbox, U, Abar, G); \
        else                                                                                                    \
            stencil_vjp_kernel<d, ns><<<g1, ADJ_BLOCK, 0, st>>>(P.gamma, limiter, N, boxes, nbox, U, Abar, G);  \
        cudaError_t e = cudaGetLastError();                                                                     \
        if (e != cudaSuccess) return e;                                                                     \
        stencil_vjp_gather<d, ns><<<g2, ADJ_BLOCK, 0, st>>>(N, boxes, nbox, G, Ubar);                       \
        return cudaGetLastError();                                                                          \
    }
    SDC_ADJ_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

template <int NS, int TOPO>
static void launch_rvjp(unsigned g, cudaStream_t st, const NetParams& P, long long N, int dim, const double* U,
                        const double* Rbar, double* Ubar, double dtm, double* rhsbar, double* abar_zone) {
    if constexpr (TOPO == TOPO_CHAIN)
        reaction_vjp_chain_kernel<NS><<<g, ADJ_BLOCK, 0, st>>>(P, N, dim, U, Rbar, Ubar, dtm, rhsbar, abar_zone);
    else
        reaction_vjp_kernel<NS, TOPO><<<g, ADJ_BLOCK, 0, st>>>(P, N, dim, U, Rbar, Ubar, dtm, rhsbar, abar_zone);
}

cudaError_t launch_reaction_vjp(const NetParams& P, int dim, long long N, const double* U, const double* Rbar,
                                double* Ubar, double dtm, double* rhsbar, double* abar_zone, cudaStream_t st) {
    const unsigned g = (unsigned)((N + ADJ_BLOCK - 1) / ADJ_BLOCK);
#define X(d, ns, tp)                                                                  \
    if (dim == d && P.nspec == ns && P.topo == tp) {                                  \
        launch_rvjp<ns, tp>(g, st, P, N, dim, U, Rbar, Ubar, dtm, rhsbar, abar_zone); \
        return cudaGetLastError();                                                    \
    }
    SDC_ADJ_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_rhs_adjoint(const RhsAdjArgs& a, cudaStream_t st) {
    if (a.N <= 0) return cudaSuccess;
    rhs_adjoint_kernel<<<(unsigned)((a.N + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reduce_rows(long long N, int rows, const double* x, double* out, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    reduce_rows_kernel<<<rows, 256, 0, st>>>(N, x, out);
    return cudaGetLastError();
}

}  // namespace sdcd
