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
//    Jacobian times the face adjoint is formed by a reverse sweep through the
//    face's operations (face_flux_vjp: one forward pass, then the adjoint of
//    each operation in reverse order, about three forward passes of work) with
//    the branches of the limiter and of HLLC fixed by the primal values, and
//    written per face; a gather adds the four face contributions of every zone
//    in a fixed order (deterministic).  face_flux_dual forms the same product
//    in forward mode (dual numbers, one input direction at a time: 4 nvar
//    passes), an independent formulation kept to cross-check the reverse one.
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

// Coefficients of the limited slope as a linear form in the three values,
// slope = cm qm + c0 q0 + cp qp, on the branch that the forward kernel's limiter
// (mc_half_slope) selects for these values: zero slope where dl and dr differ
// in sign, one is zero or |dl + dr| is below 2^-1020; else the smallest of
// |dl|, |dr|, |dl + dr|/4 (ties: |dr| over |dl|, the centred |dl + dr|/4 over
// both), compared as bit patterns on the integer pipe.
__device__ __forceinline__ void mc_slope_coef(int limiter, double qm, double q0, double qp, double& cm, double& c0,
                                              double& cp) {
    if (!limiter) { cm = -0.5; c0 = 0.0; cp = 0.5; return; }
    const double dl = q0 - qm, dr = qp - q0, s = dl + dr;
    const unsigned long long al = mag2(dl), ar = mag2(dr), as = mag2(s);
    constexpr unsigned long long E2 = (unsigned long long)EXP_ONE << 1;
    if (((dbits(dl) ^ dbits(dr)) < 0) || al == 0 || ar == 0 || as < 3 * E2) { cm = 0.0; c0 = 0.0; cp = 0.0; return; }
    const unsigned long long q = as - 2 * E2;  // |s| / 4
    const bool left = al < ar;                 // 2 dl (else 2 dr)
    const unsigned long long lim = left ? al : ar;
    if (lim < q) {
        if (left) { cm = -2.0; c0 = 2.0; cp = 0.0; }
        else { cm = 0.0; c0 = -2.0; cp = 2.0; }
    } else {                                   // slope = (dl + dr) / 2
        cm = -0.5; c0 = 0.0; cp = 0.5;
    }
}

// Ub[z][f] += (d F / d Uz[z][f])^T Fbar for the face flux of face_flux_dual:
// the same operations, differentiated by a reverse sweep.
template <int DIM, int NS>
__device__ __forceinline__ void face_flux_vjp(double gamma, int limiter, int dir, const double (*Uz)[2 + DIM + NS],
                                              const double* Fbar, double (*Ub)[2 + DIM + NS]) {
    constexpr int NV = 2 + DIM + NS;
    constexpr int IE = 1 + DIM, IX = 2 + DIM;
    const double gm1 = gamma - 1.0, igm1 = rcp_nr(gm1);
    // ---------------- forward: primitives of the four zones
    // (reciprocals and square roots by the refined forms of the forward kernel)
    double q[4][NV], irz[4];
#pragma unroll
    for (int z = 0; z < 4; z++) {
        const double rho = Uz[z][0], ir = rcp_nr(rho);
        irz[z] = ir;
        double mu = 0.0;
        q[z][0] = rho;
#pragma unroll
        for (int d = 0; d < DIM; d++) {
            const double u = Uz[z][1 + d] * ir;
            q[z][1 + d] = u;
            mu += u * Uz[z][1 + d];
        }
        q[z][IE] = gm1 * (Uz[z][IE] - 0.5 * mu);
#pragma unroll
        for (int s = 0; s < NS; s++) q[z][IX + s] = Uz[z][IX + s] * ir;
    }
    // interface states
    double qL[NV], qR[NV];
#pragma unroll
    for (int f = 0; f < NV; f++) {
        double cm, c0, cp;
        mc_slope_coef(limiter, q[0][f], q[1][f], q[2][f], cm, c0, cp);
        qL[f] = q[1][f] + 0.5 * (cm * q[0][f] + c0 * q[1][f] + cp * q[2][f]);
        mc_slope_coef(limiter, q[1][f], q[2][f], q[3][f], cm, c0, cp);
        qR[f] = q[2][f] - 0.5 * (cm * q[1][f] + c0 * q[2][f] + cp * q[3][f]);
    }
    // HLLC (Davis speeds, Toro's contact speed)
    const double rL = qL[0], rR = qR[0], unL = qL[1 + dir], unR = qR[1 + dir], pL = qL[IE], pR = qR[IE];
    double kL = 0.0, kR = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        kL += qL[1 + d] * qL[1 + d];
        kR += qR[1 + d] * qR[1 + d];
    }
    const double EL = pL * igm1 + 0.5 * rL * kL, ER = pR * igm1 + 0.5 * rR * kR;
    const double irL = rcp_nr(rL), irR = rcp_nr(rR);
    const double cL = sqrt_nr(gamma * pL * irL), cR = sqrt_nr(gamma * pR * irR);
    const bool slL = (unL - cL) <= (unR - cR);
    const double SL = slL ? unL - cL : unR - cR;
    const bool srL = (unL + cL) >= (unR + cR);
    const double SR = srL ? unL + cL : unR + cR;
    const double aL = rL * (SL - unL), aR = rR * (SR - unR);
    const double iDen = rcp_nr(aL - aR);
    const double Ss = (pR - pL + unL * aL - unR * aR) * iDen;
    const bool left = (SL >= 0.0) || (Ss >= 0.0);
    const bool star = (SL < 0.0) && (Ss >= 0.0 || SR > 0.0);
    const double* qs = left ? qL : qR;
    const double r = left ? rL : rR, un = left ? unL : unR, p = left ? pL : pR, E = left ? EL : ER;
    const double S = left ? SL : SR;
    const double ir = left ? irL : irR;
    double F0 = r * un;  // mass flux (after the star correction)
    double D = 0.0, Q = 1.0, fac = 0.0, B = 0.0, H = 0.0, iD = 0.0, iQ = 0.0;
    if (star) {
        D = r * (S - un);
        Q = S - Ss;
        iD = rcp_nr(D);
        iQ = rcp_nr(Q);
        fac = D * iQ;
        B = Ss + p * iD;
        H = E * ir + (Ss - un) * B;
        F0 += S * (fac - r);
    }
    const double* qx = (Ss >= 0.0) ? qL : qR;
    double sum = 0.0;
#pragma unroll
    for (int s = 0; s < NS; s++) sum += qx[IX + s];
    const double isum = rcp_nr(sum);

    // ---------------- reverse
    double qLb[NV], qRb[NV];
#pragma unroll
    for (int f = 0; f < NV; f++) { qLb[f] = 0.0; qRb[f] = 0.0; }
    // species: F_s = F0 X_s / sum, X from the side upwind of the contact
    double wsum = 0.0;
#pragma unroll
    for (int s = 0; s < NS; s++) wsum += Fbar[IX + s] * qx[IX + s];
    wsum *= isum;
    {
        double* qxb = (Ss >= 0.0) ? qLb : qRb;
#pragma unroll
        for (int s = 0; s < NS; s++) qxb[IX + s] += F0 * isum * (Fbar[IX + s] - wsum);
    }
    double Fhb[2 + DIM];
#pragma unroll
    for (int f = 0; f < 2 + DIM; f++) Fhb[f] = Fbar[f];
    Fhb[0] += wsum;
    double rb = 0.0, unb = 0.0, pb = 0.0, Eb = 0.0, Sb = 0.0, Ssb = 0.0, vb[DIM];
#pragma unroll
    for (int d = 0; d < DIM; d++) vb[d] = 0.0;
    if (star) {
        // F += S (Us - Uk): Us = fac (1, v with v_dir = Ss, H), Uk = (r, r v, E)
        double facb = S * Fhb[0];
        Sb += Fhb[0] * (fac - r);
        rb -= S * Fhb[0];
#pragma unroll
        for (int d = 0; d < DIM; d++) {
            const double usd = fac * (d == dir ? Ss : qs[1 + d]);
            Sb += Fhb[1 + d] * (usd - r * qs[1 + d]);
            const double usb = S * Fhb[1 + d];
            if (d == dir) { facb += usb * Ss; Ssb += usb * fac; }
            else { facb += usb * qs[1 + d]; vb[d] += usb * fac; }
            rb -= usb * qs[1 + d];
            vb[d] -= usb * r;
        }
        Sb += Fhb[IE] * (fac * H - E);
        const double ueb = S * Fhb[IE];
        Eb -= ueb;
        facb += ueb * H;
        const double Hb = ueb * fac;
        // H = E / r + (Ss - un) B,  B = Ss + p / D
        Eb += Hb * ir;
        rb -= Hb * E * (ir * ir);
        Ssb += Hb * B;
        unb -= Hb * B;
        const double Bb = Hb * (Ss - un);
        Ssb += Bb;
        pb += Bb * iD;
        double Db = -Bb * p * (iD * iD);
        // fac = D / Q,  Q = S - Ss,  D = r (S - un)
        Db += facb * iQ;
        const double Qb = -facb * fac * iQ;
        Sb += Qb;
        Ssb -= Qb;
        rb += Db * (S - un);
        Sb += Db * r;
        unb -= Db * r;
    }
    // side flux: (r un, r un v + p e_dir, (E + p) un)
    rb += Fhb[0] * un;
    unb += Fhb[0] * r;
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        rb += Fhb[1 + d] * un * qs[1 + d];
        unb += Fhb[1 + d] * r * qs[1 + d];
        vb[d] += Fhb[1 + d] * r * un;
        if (d == dir) pb += Fhb[1 + d];
    }
    Eb += Fhb[IE] * un;
    pb += Fhb[IE] * un;
    unb += Fhb[IE] * (E + p);
    unb += vb[dir];  // v_dir is un
    {
        double* qKb = left ? qLb : qRb;
        qKb[0] += rb;
        qKb[1 + dir] += unb;
#pragma unroll
        for (int d = 0; d < DIM; d++)
            if (d != dir) qKb[1 + d] += vb[d];
        qKb[IE] += pb;
    }
    double ELb = left ? Eb : 0.0, ERb = left ? 0.0 : Eb;
    double SLb = left ? Sb : 0.0, SRb = left ? 0.0 : Sb;
    // Ss = (pR - pL + unL aL - unR aR) / (aL - aR)
    {
        const double Nb = Ssb * iDen, Denb = -Ssb * Ss * iDen;
        qRb[IE] += Nb;
        qLb[IE] -= Nb;
        const double aLb = Nb * unL + Denb, aRb = -Nb * unR - Denb;
        qLb[1 + dir] += Nb * aL;
        qRb[1 + dir] -= Nb * aR;
        qLb[0] += aLb * (SL - unL);
        SLb += aLb * rL;
        qLb[1 + dir] -= aLb * rL;
        qRb[0] += aRb * (SR - unR);
        SRb += aRb * rR;
        qRb[1 + dir] -= aRb * rR;
    }
    // Davis speeds
    double cLb = 0.0, cRb = 0.0;
    if (slL) { qLb[1 + dir] += SLb; cLb -= SLb; } else { qRb[1 + dir] += SLb; cRb -= SLb; }
    if (srL) { qLb[1 + dir] += SRb; cLb += SRb; } else { qRb[1 + dir] += SRb; cRb += SRb; }
    // E = p / (gamma - 1) + r |v|^2 / 2
    qLb[IE] += ELb * igm1;
    qLb[0] += ELb * 0.5 * kL;
    qRb[IE] += ERb * igm1;
    qRb[0] += ERb * 0.5 * kR;
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        qLb[1 + d] += ELb * rL * qL[1 + d];
        qRb[1 + d] += ERb * rR * qR[1 + d];
    }
    // c = sqrt(gamma p / r)
    {
        const double tL = cLb * gamma * 0.5 * rcp_nr(cL), tR = cRb * gamma * 0.5 * rcp_nr(cR);
        qLb[IE] += tL * irL;
        qLb[0] -= tL * pL * irL * irL;
        qRb[IE] += tR * irR;
        qRb[0] -= tR * pR * irR * irR;
    }
    // interface states -> zone primitives
    double qb[4][NV];
#pragma unroll
    for (int z = 0; z < 4; z++)
#pragma unroll
        for (int f = 0; f < NV; f++) qb[z][f] = 0.0;
#pragma unroll
    for (int f = 0; f < NV; f++) {
        double cm, c0, cp;
        mc_slope_coef(limiter, q[0][f], q[1][f], q[2][f], cm, c0, cp);
        qb[0][f] += 0.5 * cm * qLb[f];
        qb[1][f] += (1.0 + 0.5 * c0) * qLb[f];
        qb[2][f] += 0.5 * cp * qLb[f];
        mc_slope_coef(limiter, q[1][f], q[2][f], q[3][f], cm, c0, cp);
        qb[1][f] -= 0.5 * cm * qRb[f];
        qb[2][f] += (1.0 - 0.5 * c0) * qRb[f];
        qb[3][f] -= 0.5 * cp * qRb[f];
    }
    // primitives -> conserved: u = m / rho, p = (gamma - 1)(E - |m|^2 / (2 rho)), X = rho X / rho
#pragma unroll
    for (int z = 0; z < 4; z++) {
        const double ir = irz[z];
        double u2 = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; d++) u2 += q[z][1 + d] * q[z][1 + d];
        const double pbz = qb[z][IE] * gm1;
        double rhob = qb[z][0] + pbz * 0.5 * u2;
#pragma unroll
        for (int d = 0; d < DIM; d++) {
            rhob -= qb[z][1 + d] * q[z][1 + d] * ir;
            Ub[z][1 + d] += qb[z][1 + d] * ir - pbz * q[z][1 + d];
        }
        Ub[z][IE] += pbz;
#pragma unroll
        for (int s = 0; s < NS; s++) {
            rhob -= qb[z][IX + s] * q[z][IX + s] * ir;
            Ub[z][IX + s] += qb[z][IX + s] * ir;
        }
        Ub[z][0] += rhob;
    }
}

}  // namespace sdcd
