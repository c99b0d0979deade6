// sdc_adjoint.cuh -- vector-Jacobian products of the SDC step (paper
// section 2, Eq. sdc:general) for its adjoint.
//
//  * Implicit reaction update: the converged root of G(w) = w - dt_m R(w) - rhs_w
//    is differentiated by the implicit-function theorem: lambda = J^-T u_w with
//    J = I - dt_m dR/dw at the root (the transposed system, dense pivoted LU),
//    d rhs_w = lambda.  R depends on rho and rho u only through T (the rates are
//    homogeneous of degree one in rho X at fixed T once the leading rho is
//    counted), so their adjoints are D_E (-E/rho + |rho u|^2/rho^2, -rho u/rho)
//    with D_E = (dR/d(rho E))^T lambda.  R is linear in every rate prefactor a_j.
//  * Advective term: A = -sum_d (F_{i+1/2} - F_{i-1/2}) / dx_d.  Every face flux
//    depends on the four zones i-1 .. i+2 along its direction; its transposed
//    Jacobian times the face adjoint is formed in forward mode (dual numbers,
//    one input direction at a time) with the branches of the limiter and of
//    HLLC fixed by the primal values, and written per face; a gather adds the
//    four face contributions of every zone in a fixed order (deterministic).
#pragma once
#include "sdc_dev.cuh"
#include "sdc_stencil.cuh"

namespace sdcd {

// value and one directional derivative
struct Dual {
    double v, d;
    __device__ Dual() : v(0.0), d(0.0) {}
    __device__ Dual(double a) : v(a), d(0.0) {}
    __device__ Dual(double a, double b) : v(a), d(b) {}
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
    const double q = a.v / b.v;
    return Dual(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ Dual dsqrt(Dual a) {
    const double s = sqrt(a.v);
    return Dual(s, a.d / (2.0 * s));
}
__device__ __forceinline__ Dual dmin(Dual a, Dual b) { return a.v <= b.v ? a : b; }
__device__ __forceinline__ Dual dmax(Dual a, Dual b) { return a.v >= b.v ? a : b; }
__device__ __forceinline__ Dual dabs(Dual a) { return a.v < 0.0 ? -a : a; }

// MC limited (or unlimited centred) slope, branches on the primal values
__device__ __forceinline__ Dual mc_slope_dual(int limiter, Dual qm, Dual q0, Dual qp) {
    const Dual dl = q0 - qm, dr = qp - q0, dc = Dual(0.5) * (dl + dr);
    if (!limiter) return dc;
    if (dl.v * dr.v <= 0.0) return Dual(0.0);
    Dual lim = dmin(Dual(2.0) * dabs(dl), Dual(2.0) * dabs(dr));
    lim = dmin(lim, dabs(dc));
    return dc.v > 0.0 ? lim : -lim;
}

// Face flux from the conserved states of the four zones around the face
// (zones l-1, l, l+1, l+2 along dir; the face lies between l and l+1).
template <int DIM, int NS>
__device__ void face_flux_dual(double gamma, int limiter, int dir, const Dual (*Uz)[2 + DIM + NS], Dual* F) {
    constexpr int NV = 2 + DIM + NS;
    const double gm1 = gamma - 1.0;
    Dual q[4][NV];
#pragma unroll
    for (int z = 0; z < 4; z++) {
        const Dual rho = Uz[z][0];
        Dual ke = Dual(0.0);
        q[z][0] = rho;
#pragma unroll
        for (int d = 0; d < DIM; d++) {
            q[z][1 + d] = Uz[z][1 + d] / rho;
            ke = ke + Dual(0.5) * rho * q[z][1 + d] * q[z][1 + d];
        }
        q[z][1 + DIM] = Dual(gm1) * (Uz[z][1 + DIM] - ke);
#pragma unroll
        for (int s = 0; s < NS; s++) q[z][2 + DIM + s] = Uz[z][2 + DIM + s] / rho;
    }
    Dual qL[NV], qR[NV];
#pragma unroll
    for (int f = 0; f < NV; f++) {
        qL[f] = q[1][f] + Dual(0.5) * mc_slope_dual(limiter, q[0][f], q[1][f], q[2][f]);
        qR[f] = q[2][f] - Dual(0.5) * mc_slope_dual(limiter, q[1][f], q[2][f], q[3][f]);
    }
    const Dual rL = qL[0], rR = qR[0];
    const Dual unL = qL[1 + dir], unR = qR[1 + dir];
    const Dual pL = qL[1 + DIM], pR = qR[1 + DIM];
    Dual kL = Dual(0.0), kR = Dual(0.0);
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        kL = kL + qL[1 + d] * qL[1 + d];
        kR = kR + qR[1 + d] * qR[1 + d];
    }
    const Dual EL = pL / Dual(gm1) + Dual(0.5) * rL * kL;
    const Dual ER = pR / Dual(gm1) + Dual(0.5) * rR * kR;
    const Dual cL = dsqrt(Dual(gamma) * pL / rL), cR = dsqrt(Dual(gamma) * pR / rR);
    const Dual SL = dmin(unL - cL, unR - cR);
    const Dual SR = dmax(unL + cL, unR + cR);
    const Dual Ss = (pR - pL + rL * unL * (SL - unL) - rR * unR * (SR - unR)) / (rL * (SL - unL) - rR * (SR - unR));
    const bool left = (SL.v >= 0.0) || (Ss.v >= 0.0);
    const bool star = (SL.v < 0.0) && (Ss.v >= 0.0 || SR.v > 0.0);
    const Dual r = left ? rL : rR, un = left ? unL : unR, p = left ? pL : pR, E = left ? EL : ER;
    const Dual S = left ? SL : SR;
    const Dual* qs = left ? qL : qR;
    Dual Fh[2 + DIM];
    Fh[0] = r * un;
#pragma unroll
    for (int d = 0; d < DIM; d++) Fh[1 + d] = r * un * qs[1 + d] + (d == dir ? p : Dual(0.0));
    Fh[1 + DIM] = (E + p) * un;
    if (star) {
        const Dual fac = r * (S - un) / (S - Ss);
        Dual Us[2 + DIM], Uk[2 + DIM];
        Us[0] = fac;
        Uk[0] = r;
#pragma unroll
        for (int d = 0; d < DIM; d++) {
            Us[1 + d] = fac * (d == dir ? Ss : qs[1 + d]);
            Uk[1 + d] = r * qs[1 + d];
        }
        Us[1 + DIM] = fac * (E / r + (Ss - un) * (Ss + p / (r * (S - un))));
        Uk[1 + DIM] = E;
#pragma unroll
        for (int f = 0; f < 2 + DIM; f++) Fh[f] = Fh[f] + S * (Us[f] - Uk[f]);
    }
#pragma unroll
    for (int f = 0; f < 2 + DIM; f++) F[f] = Fh[f];
    // species: interface X of the side upwind of the contact, renormalised
    const Dual* qx = (Ss.v >= 0.0) ? qL : qR;
    Dual sum = Dual(0.0);
#pragma unroll
    for (int s = 0; s < NS; s++) sum = sum + qx[2 + DIM + s];
#pragma unroll
    for (int s = 0; s < NS; s++) F[2 + DIM + s] = Fh[0] * (qx[2 + DIM + s] / sum);
}

}  // namespace sdcd
