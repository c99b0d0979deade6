// sdc_stencil.cuh -- advective term A(U) (paper section 2, Eq. 1: the
// divergence of the hydrodynamic fluxes) fused with the right-hand side of the
// implicit update of Eq. sdc:general.
//
// Method of lines: conserved -> primitive (rho, u, p, X), per direction a
// piecewise-linear reconstruction with MC-limited (or unlimited centred)
// slopes, interface mass fractions renormalised to sum to one, HLLC flux
// (Davis wave speeds, species flux = X of the side upwind of the contact
// times the mass flux), A = -sum_d (F_{i+1/2} - F_{i-1/2}) / dx_d.
//
// One CTA owns a TX x TY x TZ tile of one box.  The primitives of the tile
// and of its 2-zone halo along each axis (a cross-shaped region; every box is
// periodic on itself, so the halo wraps inside the box) are staged once in
// shared memory; every face flux is computed once per direction from shared
// memory and exchanged through a shared flux buffer.
#pragma once
#include "sdc_dev.cuh"

namespace sdcd {

struct BoxDev {
    long long off;  // first zone of the box in the concatenated arrays
    int n[3];
    double idx[3];  // 1/dx
};

struct TileDev {
    int box;
    int o[3];  // tile origin inside the box
};

// What the stencil kernel writes after A.
enum { STENCIL_A = 0, STENCIL_A_RHS = 1 };

// Arguments of the fused right-hand side (Eq. sdc:general, node m -> m+1):
//   rhs = U^m + dtm (A^m_new - A^m_old) - dtm R^{m+1}_old + sum_l (q_l dt) (A_l_old + R_l_old)
struct RhsArgs {
    const double* Aold[3];   // A^{(k)} at the nodes
    const double* Rold[3];   // R^{(k)} at the nodes ([n][Ntot])
    const double* Rnext;     // R^{m+1,(k)}
    const double* Aold_m;    // A^{m,(k)}
    double* rhs;
    const double* dt;        // device scalar: the step size
    double qw[3];            // q_{m,l} (units of dt)
    double dtm_frac;         // dt_m / dt
    int M;
};

__device__ __forceinline__ double mc_slope(int limiter, double qm, double q0, double qp) {
    const double dl = q0 - qm, dr = qp - q0, dc = 0.5 * (dl + dr);
    if (!limiter) return dc;
    if (dl * dr <= 0.0) return 0.0;
    double lim = fmin(2.0 * fabs(dl), 2.0 * fabs(dr));
    lim = fmin(lim, fabs(dc));
    return dc > 0.0 ? lim : -lim;
}

// HLLC flux through a face normal to `dir`; q = [rho, u_0.., p, X_0..].
template <int DIM, int NS>
__device__ __forceinline__ void hllc_flux(double g, double gm1_inv, int dir, const double* qL, const double* qR,
                                          double* F) {
    const double rL = qL[0], rR = qR[0];
    const double unL = qL[1 + dir], unR = qR[1 + dir];
    const double pL = qL[1 + DIM], pR = qR[1 + DIM];
    double kL = 0.0, kR = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        kL += qL[1 + d] * qL[1 + d];
        kR += qR[1 + d] * qR[1 + d];
    }
    const double EL = pL * gm1_inv + 0.5 * rL * kL;
    const double ER = pR * gm1_inv + 0.5 * rR * kR;
    const double cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
    const double SL = fmin(unL - cL, unR - cR);
    const double SR = fmax(unL + cL, unR + cR);
    const double Ss = (pR - pL + rL * unL * (SL - unL) - rR * unR * (SR - unR)) /
                      (rL * (SL - unL) - rR * (SR - unR));
    // region: SL >= 0 -> F_L; else Ss >= 0 -> F*_L; else SR > 0 -> F*_R; else F_R
    const bool left = (SL >= 0.0) || (Ss >= 0.0);
    const bool star = (SL < 0.0) && (Ss >= 0.0 || SR > 0.0);
    const double r = left ? rL : rR, un = left ? unL : unR, p = left ? pL : pR, E = left ? EL : ER;
    const double S = left ? SL : SR;
    const double* q = left ? qL : qR;
    const double* qx = (Ss >= 0.0) ? qL : qR;  // species: side upwind of the contact
    double Fh[2 + DIM];
    Fh[0] = r * un;
#pragma unroll
    for (int d = 0; d < DIM; d++) Fh[1 + d] = r * un * q[1 + d] + (d == dir ? p : 0.0);
    Fh[1 + DIM] = (E + p) * un;
    if (star) {
        const double fac = r * (S - un) / (S - Ss);
        double Us[2 + DIM];
        Us[0] = fac;
#pragma unroll
        for (int d = 0; d < DIM; d++) Us[1 + d] = fac * (d == dir ? Ss : q[1 + d]);
        Us[1 + DIM] = fac * (E / r + (Ss - un) * (Ss + p / (r * (S - un))));
        double Uk[2 + DIM];
        Uk[0] = r;
#pragma unroll
        for (int d = 0; d < DIM; d++) Uk[1 + d] = r * q[1 + d];
        Uk[1 + DIM] = E;
#pragma unroll
        for (int f = 0; f < 2 + DIM; f++) Fh[f] = Fh[f] + S * (Us[f] - Uk[f]);
    }
#pragma unroll
    for (int f = 0; f < 2 + DIM; f++) F[f] = Fh[f];
#pragma unroll
    for (int s = 0; s < NS; s++) F[2 + DIM + s] = Fh[0] * qx[2 + DIM + s];
}

template <int DIM, int TX, int TY, int TZ>
struct TileGeom {
    static constexpr int HX = TX + 4;
    static constexpr int NXE = HX * TY * TZ;                 // x-extended slab
    static constexpr int NYH = (DIM >= 2) ? TX * 4 * TZ : 0;  // y halo slabs
    static constexpr int NZH = (DIM >= 3) ? TX * TY * 4 : 0;  // z halo slabs
    static constexpr int NC = NXE + NYH + NZH;
    static constexpr int FX = (TX + 1) * TY * TZ;
    static constexpr int FY = (DIM >= 2) ? TX * (TY + 1) * TZ : 0;
    static constexpr int FZ = (DIM >= 3) ? TX * TY * (TZ + 1) : 0;
    static constexpr int NF = FX > FY ? (FX > FZ ? FX : FZ) : (FY > FZ ? FY : FZ);
    static constexpr int NT = TX * TY * TZ;
};

// shared-memory slot of tile-local zone (x, y, z); at most one coordinate
// lies outside the tile extents (ex, ey, ez)
template <int DIM, int TX, int TY, int TZ>
__device__ __forceinline__ int slot_of(int x, int y, int z, int ey, int ez) {
    using G = TileGeom<DIM, TX, TY, TZ>;
    if (DIM >= 2 && (y < 0 || y >= ey)) {
        const int ys = y < 0 ? y + 2 : y - ey + 2;
        return G::NXE + x + TX * (ys + 4 * z);
    }
    if (DIM >= 3 && (z < 0 || z >= ez)) {
        const int zs = z < 0 ? z + 2 : z - ez + 2;
        return G::NXE + G::NYH + x + TX * (y + TY * zs);
    }
    return (x + 2) + G::HX * (y + TY * z);
}

__device__ __forceinline__ int wrap(int g, int n) {
    g %= n;
    return g < 0 ? g + n : g;
}

template <int DIM, int NS, int TX, int TY, int TZ, int MODE>
__global__ void __launch_bounds__(TX * TY * TZ)
stencil_kernel(NetParams P, int limiter, long long Ntot, const BoxDev* __restrict__ boxes,
               const TileDev* __restrict__ tiles, const double* __restrict__ U, double* __restrict__ Aout,
               RhsArgs ra) {
    using G = TileGeom<DIM, TX, TY, TZ>;
    constexpr int NV = 2 + DIM + NS;
    extern __shared__ double smem[];
    double* sq = smem;                 // [NV][NC] primitives
    double* sf = smem + NV * G::NC;    // [NV][NF] face fluxes of one direction

    const TileDev t = tiles[blockIdx.x];
    const BoxDev b = boxes[t.box];
    const int ex = min(TX, b.n[0] - t.o[0]);
    const int ey = DIM >= 2 ? min(TY, b.n[1] - t.o[1]) : 1;
    const int ez = DIM >= 3 ? min(TZ, b.n[2] - t.o[2]) : 1;
    const double g = P.gamma, gm1 = P.gm1, gm1_inv = 1.0 / P.gm1;

    // ---- stage primitives of the tile and its cross-shaped halo
    for (int s = threadIdx.x; s < G::NC; s += blockDim.x) {
        int x, y, z;
        if (s < G::NXE) {
            x = s % G::HX - 2;
            const int r = s / G::HX;
            y = r % TY;
            z = r / TY;
            if (x >= ex + 2 || y >= ey || z >= ez) continue;
        } else if (DIM >= 2 && s < G::NXE + G::NYH) {
            const int i = s - G::NXE;
            x = i % TX;
            const int r = i / TX;
            const int ys = r % 4;
            z = r / 4;
            y = ys < 2 ? ys - 2 : ey + ys - 2;
            if (x >= ex || z >= ez) continue;
        } else {
            const int i = s - G::NXE - G::NYH;
            x = i % TX;
            const int r = i / TX;
            y = r % TY;
            const int zs = r / TY;
            z = zs < 2 ? zs - 2 : ez + zs - 2;
            if (x >= ex || y >= ey) continue;
        }
        const int gx = wrap(t.o[0] + x, b.n[0]);
        const int gy = DIM >= 2 ? wrap(t.o[1] + y, b.n[1]) : 0;
        const int gz = DIM >= 3 ? wrap(t.o[2] + z, b.n[2]) : 0;
        const long long gi = b.off + gx + (long long)b.n[0] * (gy + (long long)b.n[1] * gz);
        const double rho = __ldg(U + gi);
        const double ir = 1.0 / rho;
        double ke = 0.0;
        sq[0 * G::NC + s] = rho;
#pragma unroll
        for (int d = 0; d < DIM; d++) {
            const double u = __ldg(U + (1 + d) * Ntot + gi) * ir;
            sq[(1 + d) * G::NC + s] = u;
            ke += 0.5 * rho * u * u;
        }
        sq[(1 + DIM) * G::NC + s] = gm1 * (__ldg(U + (1 + DIM) * Ntot + gi) - ke);
#pragma unroll
        for (int sp = 0; sp < NS; sp++) sq[(2 + DIM + sp) * G::NC + s] = __ldg(U + (2 + DIM + sp) * Ntot + gi) * ir;
    }
    __syncthreads();

    // zone owned by this thread
    const int tx = threadIdx.x % TX, ty = (threadIdx.x / TX) % TY, tz = threadIdx.x / (TX * TY);
    const bool own = (threadIdx.x < G::NT) && tx < ex && ty < ey && tz < ez;
    double A[NV];
#pragma unroll
    for (int f = 0; f < NV; f++) A[f] = 0.0;

#pragma unroll
    for (int dir = 0; dir < DIM; dir++) {
        // faces of this direction: position i in [0, e_dir] along dir (face i sits
        // between zones i-1 and i), the other two coordinates inside the tile
        const int e0 = dir == 0 ? ex + 1 : ex;
        const int e1 = dir == 1 ? ey + 1 : ey;
        const int e2 = dir == 2 ? ez + 1 : ez;
        const int T0 = dir == 0 ? TX + 1 : TX;
        const int T1 = dir == 1 ? TY + 1 : TY;
        const int nfaces = T0 * T1 * (dir == 2 ? TZ + 1 : TZ);
        for (int fi = threadIdx.x; fi < nfaces; fi += blockDim.x) {
            const int c0 = fi % T0, c1 = (fi / T0) % T1, c2 = fi / (T0 * T1);
            if (c0 >= e0 || c1 >= e1 || c2 >= e2) continue;
            int sl[4];
#pragma unroll
            for (int o = 0; o < 4; o++) {
                int c[3] = {c0, c1, c2};
                c[dir] += o - 2;
                sl[o] = slot_of<DIM, TX, TY, TZ>(c[0], c[1], c[2], ey, ez);
            }
            double qL[NV], qR[NV];
#pragma unroll
            for (int f = 0; f < NV; f++) {
                const double a0 = sq[f * G::NC + sl[0]], a1 = sq[f * G::NC + sl[1]];
                const double a2 = sq[f * G::NC + sl[2]], a3 = sq[f * G::NC + sl[3]];
                qL[f] = a1 + 0.5 * mc_slope(limiter, a0, a1, a2);
                qR[f] = a2 - 0.5 * mc_slope(limiter, a1, a2, a3);
            }
            if (NS > 0) {
                double sL = 0.0, sR = 0.0;
#pragma unroll
                for (int s = 0; s < NS; s++) { sL += qL[2 + DIM + s]; sR += qR[2 + DIM + s]; }
                const double iL = 1.0 / sL, iR = 1.0 / sR;
#pragma unroll
                for (int s = 0; s < NS; s++) { qL[2 + DIM + s] *= iL; qR[2 + DIM + s] *= iR; }
            }
            double F[NV];
            hllc_flux<DIM, NS>(g, gm1_inv, dir, qL, qR, F);
#pragma unroll
            for (int f = 0; f < NV; f++) sf[f * G::NF + fi] = F[f];
        }
        __syncthreads();
        if (own) {
            int c[3] = {tx, ty, tz};
            const int T0s = dir == 0 ? TX + 1 : TX, T1s = dir == 1 ? TY + 1 : TY;
            const int lo = c[0] + T0s * (c[1] + T1s * c[2]);
            c[dir] += 1;
            const int hi = c[0] + T0s * (c[1] + T1s * c[2]);
            const double idx = b.idx[dir];
#pragma unroll
            for (int f = 0; f < NV; f++) A[f] -= (sf[f * G::NF + hi] - sf[f * G::NF + lo]) * idx;
        }
        __syncthreads();
    }

    if (!own) return;
    const long long gi = b.off + (t.o[0] + tx) + (long long)b.n[0] * ((t.o[1] + ty) + (long long)b.n[1] * (t.o[2] + tz));
#pragma unroll
    for (int f = 0; f < NV; f++) Aout[f * Ntot + gi] = A[f];
    if (MODE == STENCIL_A_RHS) {
        const double dt = *ra.dt;
        const double dtm = dt * ra.dtm_frac;
        double qdt[3];
#pragma unroll
        for (int l = 0; l < 3; l++) qdt[l] = ra.qw[l] * dt;
#pragma unroll
        for (int f = 0; f < NV; f++) {
            double v = __ldg(U + f * Ntot + gi) + dtm * (A[f] - __ldg(ra.Aold_m + f * Ntot + gi));
            const bool reactive = f >= 1 + DIM;
            const int r = f - 1 - DIM;
            if (reactive) v -= dtm * __ldg(ra.Rnext + r * Ntot + gi);
            double I = 0.0;
            for (int l = 0; l < ra.M; l++) {
                double src = __ldg(ra.Aold[l] + f * Ntot + gi);
                if (reactive) src += __ldg(ra.Rold[l] + r * Ntot + gi);
                I += qdt[l] * src;
            }
            ra.rhs[f * Ntot + gi] = v + I;
        }
    }
}

}  // namespace sdcd
