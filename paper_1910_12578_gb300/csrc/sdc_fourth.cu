// sdc_fourth.cu -- fourth-order finite-volume operators of the SDC step
// (paper section 2: the fourth-order method pairs Simpson's rule with the
// spatial reconstruction of McCorquodale & Colella), smooth-flow form without
// limiting.  With L the sum over the box's dimensions of second differences:
//   zone centres and averages:  f_c = <f> - L<f>/24,  <f> = f_c + L f_c/24;
//   primitive averages          <W> = W(U_c) + L W(<U>)/24;
//   face averages               <W>_{i+1/2} = 7/12 (<W>_i + <W>_{i+1})
//                                           - 1/12 (<W>_{i-1} + <W>_{i+2});
//   face-centre states          W_f = <W>_{i+1/2} - L_t <W>_{i+1/2}/24
//                               (L_t: second differences across the face);
//   face-average fluxes         <F> = F(W_f) + L_t F(<W>_{i+1/2})/24;
//   A = -sum_d (<F>_{i+1/2} - <F>_{i-1/2}) / dx_d.
// Both sides of a face see the same state, so F is the physical Euler flux.
// Limited form (limiter 1): a face average outside the range of its two zone
// averages is replaced by their mean less a sixth of a limited second
// difference (Colella & Sekora's face limiter); then every zone limits its two
// face values, by a limited curvature at an extremum (of the face values about
// the average, or of the averages at distance one or two, with differences of
// rounding size counting as ties) and by the PPM
// overshoot bounds elsewhere; the limited mass fractions are renormalised; the
// two sides of a face then give its flux by HLLC, at the face centres and from
// the face averages alike.  The averaged source is R(U_c) + L R(U_c)/24; the implicit update is solved at
// zone centres (U_c - dt_m R(U_c) = rhs_c) and gives <U> = <rhs> + dt_m <R>.
// Every operator is a sequence of elementwise kernels over field-major arrays,
// one thread per zone, periodic within each box.  GB300 issues FP64 at 2 lanes
// per SM per clock, so even these stencils are bound by the FP64 pipe: the
// kernels divide once per zone (a refined hardware reciprocal) and multiply.
#include "sdc_fourth_launch.h"
#include "sdc_launch.h"

namespace sdcd {
namespace {

constexpr int F_BLOCK = 256;

inline unsigned fgrid(long long n) { return (unsigned)((n + F_BLOCK - 1) / F_BLOCK); }

__device__ __forceinline__ int box_index(const BoxDev* boxes, int nbox, long long z) {
    int lo = 0, hi = nbox - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (boxes[mid].off <= z) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// zone-local coordinates of z inside its box
struct ZoneCoord {
    long long off;
    int n[3], c[3];
};

__device__ __forceinline__ ZoneCoord zone_coord(const BoxDev* boxes, int nbox, long long z) {
    const BoxDev b = boxes[box_index(boxes, nbox, z)];
    ZoneCoord q;
    q.off = b.off;
    for (int d = 0; d < 3; d++) q.n[d] = b.n[d];
    // 32-bit arithmetic inside the box (fewer than 2^31 zones): 64-bit division
    // would run on the narrow FP64 pipe
    const int l = (int)(z - b.off);
    q.c[0] = l % b.n[0];
    q.c[1] = (l / b.n[0]) % b.n[1];
    q.c[2] = l / (b.n[0] * b.n[1]);
    return q;
}

// zone indices o steps from z along d, periodic in the box (|o| <= 2, any n >= 1)
struct Line {
    long long z, stride;
    int c, n;
    __device__ __forceinline__ long long at(int o) const {
        int cc = c + o;
        while (cc < 0) cc += n;
        while (cc >= n) cc -= n;
        return z + (long long)(cc - c) * stride;
    }
};

// element d of a 3-array by selects (a runtime index would put the array on the stack)
__device__ __forceinline__ int sel3(const int* a, int d) { return d == 0 ? a[0] : (d == 1 ? a[1] : a[2]); }

__device__ __forceinline__ Line line_of(const ZoneCoord& q, long long z, int d) {
    Line l;
    l.z = z;
    l.c = sel3(q.c, d);
    l.n = sel3(q.n, d);
    l.stride = d == 0 ? 1 : (d == 1 ? (long long)q.n[0] : (long long)q.n[0] * q.n[1]);
    return l;
}

// neighbours of z along the dimensions d < dim other than skip (skip = -1: all),
// as scalars (an index array over a runtime dimension count would sit on the
// stack), and -2 n_d
struct LapNb {
    long long p0, m0, p1, m1, p2, m2;
    bool u0, u1, u2;
    double c2;
};

__device__ __forceinline__ LapNb lap_nb(const ZoneCoord& q, long long z, int dim, int skip) {
    LapNb nb;
    nb.u0 = 0 < dim && skip != 0;
    nb.u1 = 1 < dim && skip != 1;
    nb.u2 = 2 < dim && skip != 2;
    nb.p0 = nb.m0 = nb.p1 = nb.m1 = nb.p2 = nb.m2 = z;
    if (nb.u0) {
        const Line l = line_of(q, z, 0);
        nb.p0 = l.at(1);
        nb.m0 = l.at(-1);
    }
    if (nb.u1) {
        const Line l = line_of(q, z, 1);
        nb.p1 = l.at(1);
        nb.m1 = l.at(-1);
    }
    if (nb.u2) {
        const Line l = line_of(q, z, 2);
        nb.p2 = l.at(1);
        nb.m2 = l.at(-1);
    }
    nb.c2 = -2.0 * (int(nb.u0) + int(nb.u1) + int(nb.u2));
    return nb;
}

// a + coef * sum_d (b(z+e_d) - 2 b(z) + b(z-e_d)) for one field (offset o), formed
// as a + coef (sum of the neighbour pairs - 2 n_d b(z)): one add per neighbour,
// then two FMAs (the FP64 pipe is the bound)
__device__ __forceinline__ double lap_at(const double* __restrict__ b, long long o, long long z, const LapNb& nb,
                                         double a, double coef) {
    double sn = 0.0;
    bool first = true;
    if (nb.u0) {
        sn = b[o + nb.p0] + b[o + nb.m0];
        first = false;
    }
    if (nb.u1) {
        const double pair = b[o + nb.p1] + b[o + nb.m1];
        sn = first ? pair : sn + pair;
        first = false;
    }
    if (nb.u2) {
        const double pair = b[o + nb.p2] + b[o + nb.m2];
        sn = first ? pair : sn + pair;
    }
    return fma(coef, fma(nb.c2, b[o + z], sn), a);
}

// out = a + coef * sum_{d < dim, d != skip} (b(z+e_d) - 2 b(z) + b(z-e_d)), nf fields
__global__ void lap_combine_kernel(int dim, int nf, long long N, const BoxDev* __restrict__ boxes, int nbox,
                                   const double* __restrict__ a, const double* __restrict__ b, double coef, int skip,
                                   double* __restrict__ out) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const LapNb nb = lap_nb(zone_coord(boxes, nbox, z), z, dim, skip);
    for (int f = 0; f < nf; f++) {
        const long long o = (long long)f * N;
        out[o + z] = lap_at(b, o, z, nb, a[o + z], coef);
    }
}

// out1 = b1 + coef L b1 and out2 = b2 + coef L b2 (two maps over one index set)
__global__ void lap_pair_kernel(int dim, int nf, long long N, const BoxDev* __restrict__ boxes, int nbox,
                                const double* __restrict__ b1, double* __restrict__ out1,
                                const double* __restrict__ b2, double* __restrict__ out2, double coef) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const LapNb nb = lap_nb(zone_coord(boxes, nbox, z), z, dim, -1);
    for (int f = 0; f < nf; f++) {
        const long long o = (long long)f * N;
        out1[o + z] = lap_at(b1, o, z, nb, b1[o + z], coef);
        out2[o + z] = lap_at(b2, o, z, nb, b2[o + z], coef);
    }
}

// Wc = W(U_c) with U_c = U - L U/24 formed field by field as it is needed, and
// W2 = W(U) = (rho, m/rho, (gamma-1)(E - m.u/2), rho X/rho): the centre map and
// both primitive conversions in one pass, one reciprocal of rho each
__global__ void prims4_kernel(int dim, int nspec, double gm1, long long N, const BoxDev* __restrict__ boxes, int nbox,
                              const double* __restrict__ U, double* __restrict__ Wc, double* __restrict__ W2) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const LapNb nb = lap_nb(zone_coord(boxes, nbox, z), z, dim, -1);
    constexpr double c24 = -1.0 / 24.0;
    const double rho = U[z], ir = rcp_nr(rho);
    const double rc = lap_at(U, 0, z, nb, rho, c24), irc = rcp_nr(rc);
    W2[z] = rho;
    Wc[z] = rc;
    double ke = 0.0, kec = 0.0;
    for (int d = 0; d < dim; d++) {
        const long long o = (long long)(1 + d) * N;
        const double m = U[o + z], u = m * ir;
        const double mc = lap_at(U, o, z, nb, m, c24), uc = mc * irc;
        W2[o + z] = u;
        Wc[o + z] = uc;
        ke += 0.5 * m * u;
        kec += 0.5 * mc * uc;
    }
    {
        const long long o = (long long)(1 + dim) * N;
        const double E = U[o + z];
        W2[o + z] = gm1 * (E - ke);
        Wc[o + z] = gm1 * (lap_at(U, o, z, nb, E, c24) - kec);
    }
    for (int s = 0; s < nspec; s++) {
        const long long o = (long long)(2 + dim + s) * N;
        const double v = U[o + z];
        W2[o + z] = v * ir;
        Wc[o + z] = lap_at(U, o, z, nb, v, c24) * irc;
    }
}

// face averages of the primitives, the face between z and its +1 neighbour along dir
__global__ void face_avg_kernel(int dir, int nf, long long N, const BoxDev* __restrict__ boxes, int nbox,
                                const double* __restrict__ Wa, double* __restrict__ Wf) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const ZoneCoord q = zone_coord(boxes, nbox, z);
    const Line l = line_of(q, z, dir);
    const long long zm = l.at(-1), zp = l.at(1), zpp = l.at(2);
    for (int f = 0; f < nf; f++) {
        const long long o = (long long)f * N;
        Wf[o + z] = 7.0 / 12.0 * (Wa[o + z] + Wa[o + zp]) - 1.0 / 12.0 * (Wa[o + zm] + Wa[o + zpp]);
    }
}

// Fc = F(Wfc) (face centres), F2 = F(Wf) (from the face averages): the physical
// Euler flux along dir, hydrodynamic fields in registers, species streamed
// (mass flux times X)
template <int DIM>
__global__ void face_flux_kernel(int nspec, double igm1, int dir, long long N, const double* __restrict__ Wfc,
                                 const double* __restrict__ Wf, double* __restrict__ Fc, double* __restrict__ F2) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    constexpr int NH = 2 + DIM;
    const int nv = NH + nspec;
#pragma unroll
    for (int side = 0; side < 2; side++) {
        const double* W = side ? Wf : Wfc;
        double* F = side ? F2 : Fc;
        double qv[NH];
#pragma unroll
        for (int f = 0; f < NH; f++) qv[f] = W[(long long)f * N + z];
        const double rho = qv[0], p = qv[1 + DIM];
        double un = qv[1];
#pragma unroll
        for (int d = 1; d < DIM; d++)
            if (d == dir) un = qv[1 + d];
        double k2 = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; d++) k2 = fma(qv[1 + d], qv[1 + d], k2);
        const double E = fma(p, igm1, 0.5 * rho * k2);
        F[z] = rho * un;
#pragma unroll
        for (int d = 0; d < DIM; d++) F[(long long)(1 + d) * N + z] = rho * un * qv[1 + d] + (d == dir ? p : 0.0);
        F[(long long)(1 + DIM) * N + z] = (E + p) * un;
        for (int f = NH; f < nv; f++) F[(long long)f * N + z] = rho * un * W[(long long)f * N + z];
    }
}

// ---- limited form
constexpr double CS_C = 1.25;  // bound of the limited curvature over its neighbours'

// Sign tests on bit patterns (integer pipe; FP64 compares and products issue on
// the narrow FP64 pipe).  They equal the plain products' tests except when a
// product of two nonzero differences underflows to zero.
__device__ __forceinline__ bool nonzero(double x) { return mag2(x) != 0ull; }
// x y < 0
__device__ __forceinline__ bool opposite(double x, double y) {
    return nonzero(x) && nonzero(y) && (dbits(x) ^ dbits(y)) < 0;
}
// x y > 0
__device__ __forceinline__ bool same2(double x, double y) {
    return nonzero(x) && nonzero(y) && (dbits(x) ^ dbits(y)) >= 0;
}
// of two values of one sign, the smaller in magnitude
__device__ __forceinline__ double min_mag(double x, double y) { return mag2(x) <= mag2(y) ? x : y; }

// face between zones a0 and ap (neighbours am, app) whose value af lies outside
// [a0, ap]: it becomes (a0 + ap)/2 - d2/6, d2 the second difference
// 3 (a0 - 2 af + ap) limited by C times those of the two zones (0 unless all
// three share a sign); the unlimited d2 would return af itself
__device__ __forceinline__ double cs_face_limit(double am, double a0, double ap, double app, double af) {
    const double d2f = 3.0 * fma(-2.0, af, a0 + ap);
    const double d2l = fma(-2.0, a0, am + ap), d2r = fma(-2.0, ap, a0 + app);
    double d2 = 0.0;
    if (same2(d2f, d2l) && same2(d2f, d2r)) d2 = min_mag(d2f, CS_C * min_mag(d2l, d2r));
    return fma(d2, -1.0 / 6.0, 0.5 * (a0 + ap));
}

// The extremum tests compare the signs of two differences of averages on
// either side of the zone, e = a_left - a0 and e' = a0 - a_right.  Averages
// mirrored across a plane of symmetry of the data differ only by rounding, and
// a test would take its branch from the order of that rounding: a difference
// counts as zero (a tie) when it is at most 2^-20 of the other one or at most
// 2^-48 of the larger average it is formed from.  2^-k |x| is the bit pattern
// of x less k in the exponent field (mag2 units of 2^53); where that leaves the
// normal range only an exact zero counts.
__device__ __forceinline__ double tie_diff(double d, double other, double a, double b) {
    constexpr unsigned long long R20 = 20ull << 53, A48 = 48ull << 53;
    const unsigned long long md = mag2(d), mo = mag2(other), M = max(mag2(a), mag2(b));
    if (md <= (mo > R20 ? mo - R20 : 0ull)) return 0.0;
    if (md <= (M > A48 ? M - A48 : 0ull)) return 0.0;
    return d;
}

// Zone limiter of zone a0 (neighbours amm .. app) with face values fm, fp and
// their deviations dm = fm - a0, dp = fp - a0 (limit4_kernel): an extremum when
// the deviations do not have opposite signs or the differences e1 = am - a0,
// e2 = a0 - ap (or e3 = amm - a0, e4 = a0 - app) are not of one sign after the
// tie rule of tie_diff; there both deviations are scaled by the limited
// curvature over the parabola's (cs_zone_extremum; the centred second
// differences come from the differences above: they enter only through signs
// and magnitudes, where the limiter is continuous, so a curvature near zero
// flattens either way); elsewhere (dm, dp nonzero) the parabola may not
// overshoot the far face: |dp| >= 2 |dm| on the bit patterns (2 |dm| is |dm|
// with the exponent field raised by one; subnormal dm aside) sets fp = a0 - 2 dm,
// and the same the other way.

// The zone limiter's extremum branch for one (zone, field): the two deviations
// scaled by the limited curvature over the parabola's (the zone limiter above);
// e1..e4 the differences of the extremum tests.
__device__ __forceinline__ void cs_zone_extremum(double a0, double dm, double dp, double e1, double e2, double e3,
                                                 double e4, double& fm, double& fp) {
    const double d2 = 6.0 * (dm + dp);
    const double d2c = e1 - e2, d2l = fma(-2.0, e1, e3), d2r = fma(2.0, e2, -e4);
    if (same2(d2, d2c) && same2(d2, d2l) && same2(d2, d2r)) {
        const double cm = CS_C * min_mag(d2c, min_mag(d2l, d2r));
        if (mag2(d2) <= mag2(cm)) {
            fm = a0 + dm;
            fp = a0 + dp;
        } else {
            // in (0, 1); the refined reciprocal takes normal d2 only
            // (2^-1021 <= |d2| < 2^1022), the division the rest
            const unsigned long long ex = mag2(d2) >> 53;
            const double sc = (ex >= 2ull && ex < 2045ull) ? cm * rcp_nr(d2) : cm / d2;
            fm = fma(dm, sc, a0);
            fp = fma(dp, sc, a0);
        }
    } else {
        fm = a0;
        fp = a0;
    }
}

// One thread per zone: the zone's two face averages along dir from the
// primitive averages z-2 .. z+2, each through the face limiter, then both
// through the zone limiter; WL[z] = the upper face (left side of the face
// z+1/2), WR[z-1] = the lower face (right side of the face z-1/2).  The limited
// mass fractions are renormalised: stored first, then read back and scaled.
// The face tests' differences give the deviations dm, dp when no face limiter
// fires (fm - a0 = -(a0 - fm) exactly).
//
// The zone limiter's extremum branch (curvatures, their limited minimum and a
// reciprocal) is taken by a scattered minority of (zone, field) pairs, which
// would make most warps issue it for a few lanes field after field.  Instead a
// lane whose field needs it queues the field's inputs in its warp's shared
// queue; whenever 32 items are waiting, the warp's lanes take one each, and the
// rest is drained at the end.  The arithmetic per (zone, field) is that of
// the zone limiter above wherever a lane computes it, so the results do not
// depend on the queue.
constexpr int LIM_Q = 64;   // queue slots per warp (at most 31 waiting + 32 arriving)
__global__ void __launch_bounds__(F_BLOCK)
limit4_kernel(int dim, int nspec, int dir, long long N, const BoxDev* __restrict__ boxes, int nbox,
              const double* __restrict__ Wa, double* __restrict__ WL, double* __restrict__ WR) {
    __shared__ double qv[F_BLOCK / 32][7][LIM_Q];   // a0, dm, dp, e1, e2, e3, e4
    __shared__ long long qz[F_BLOCK / 32][2][LIM_Q];  // the owner's zone index z and lower neighbour i1
    __shared__ int qf[F_BLOCK / 32][LIM_Q];           // the field
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = z < N;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    long long i0 = z, i1 = z, i3 = z, i4 = z;
    if (act) {
        const ZoneCoord q = zone_coord(boxes, nbox, z);
        const Line l = line_of(q, z, dir);
        i0 = l.at(-2); i1 = l.at(-1); i3 = l.at(1); i4 = l.at(2);
    }
    const int nh = 2 + dim, nv = nh + nspec;
    int cnt = 0;  // items waiting in the warp's queue (the same in every lane)
    auto drain = [&](int n) {
        // lanes 0..n-1 take items 0..n-1
        if (lane < n) {
            double fm, fp;
            const double a0 = qv[wq][0][lane];
            cs_zone_extremum(a0, qv[wq][1][lane], qv[wq][2][lane], qv[wq][3][lane], qv[wq][4][lane],
                             qv[wq][5][lane], qv[wq][6][lane], fm, fp);
            const long long o = (long long)qf[wq][lane] * N;
            WL[o + qz[wq][0][lane]] = fp;
            WR[o + qz[wq][1][lane]] = fm;
        }
        __syncwarp();
    };
    for (int f = 0; f < nv; f++) {
        const long long o = (long long)f * N;
        bool ext = false;
        double a0 = 0.0, dm = 0.0, dp = 0.0, e1 = 0.0, e2 = 0.0, e3 = 0.0, e4 = 0.0;
        if (act) {
            const double amm = Wa[o + i0], am = Wa[o + i1], ap = Wa[o + i3], app = Wa[o + i4];
            a0 = Wa[o + z];
            double fm = 7.0 / 12.0 * (am + a0) - 1.0 / 12.0 * (amm + ap);
            double fp = 7.0 / 12.0 * (a0 + ap) - 1.0 / 12.0 * (am + app);
            // face tests: (af - left)(right - af) < 0 puts af outside its zones' range
            double lo = a0 - fm;  // -dm
            if (opposite(fm - am, lo)) {
                fm = cs_face_limit(amm, am, a0, ap, fm);
                lo = a0 - fm;
            }
            dp = fp - a0;
            if (opposite(dp, ap - fp)) {
                fp = cs_face_limit(am, a0, ap, app, fp);
                dp = fp - a0;
            }
            dm = -lo;
            // the zone limiter: the extremum tests, then the monotone
            // branch here or the extremum branch through the queue
            e1 = am - a0; e2 = a0 - ap; e3 = amm - a0; e4 = a0 - app;
            const double t1 = tie_diff(e1, e2, am, a0), t2 = tie_diff(e2, e1, a0, ap);
            const double t3 = tie_diff(e3, e4, amm, a0), t4 = tie_diff(e4, e3, a0, app);
            ext = !opposite(dp, dm) || !same2(t1, t2) || !same2(t3, t4);
            if (!ext) {
                constexpr unsigned long long E1 = 1ull << 53;
                if (mag2(dp) >= mag2(dm) + E1) fp = fma(-2.0, dm, a0);
                if (mag2(dm) >= mag2(dp) + E1) fm = fma(-2.0, dp, a0);
                WL[o + z] = fp;
                WR[o + i1] = fm;
            }
        }
        const unsigned b = __ballot_sync(0xffffffffu, ext);
        if (ext) {
            const int slot = cnt + __popc(b & lt);
            qv[wq][0][slot] = a0; qv[wq][1][slot] = dm; qv[wq][2][slot] = dp;
            qv[wq][3][slot] = e1; qv[wq][4][slot] = e2; qv[wq][5][slot] = e3; qv[wq][6][slot] = e4;
            qz[wq][0][slot] = z; qz[wq][1][slot] = i1;
            qf[wq][slot] = f;
        }
        cnt += __popc(b);
        __syncwarp();
        if (cnt >= 32) {
            drain(32);
            // the waiting rest moves to the front
            const int rest = cnt - 32;
            if (lane < rest) {
                for (int v = 0; v < 7; v++) qv[wq][v][lane] = qv[wq][v][32 + lane];
                qz[wq][0][lane] = qz[wq][0][32 + lane];
                qz[wq][1][lane] = qz[wq][1][32 + lane];
                qf[wq][lane] = qf[wq][32 + lane];
            }
            __syncwarp();
            cnt = rest;
        }
    }
    if (cnt > 0) drain(cnt);
    // renormalised mass fractions: the sums in field order, as written
    if (act && nspec > 0) {
        double sm = 0.0, sp = 0.0;
        for (int f = nh; f < nv; f++) {
            const long long o = (long long)f * N;
            sm += WR[o + i1];
            sp += WL[o + z];
        }
        const double rm = 1.0 / sm, rp = 1.0 / sp;
        for (int f = nh; f < nv; f++) {
            const long long o = (long long)f * N;
            WL[o + z] *= rp;
            WR[o + i1] *= rm;
        }
    }
}

// transverse neighbours of z (the dimensions other than dir): up to 2 pairs
struct Transverse {
    long long p[2], m[2];
    int nt;
};

__device__ __forceinline__ Transverse transverse_of(const ZoneCoord& q, long long z, int dim, int dir) {
    // the dimensions other than dir, ascending: (1, 2), (0, 2) or (0, 1)
    const int d1 = dir == 0 ? 1 : 0, d2 = dir == 2 ? 1 : 2;
    Transverse t;
    t.nt = (d1 < dim) + (d2 < dim);
    t.p[0] = t.m[0] = t.p[1] = t.m[1] = z;
    if (d1 < dim) {
        const Line l = line_of(q, z, d1);
        t.p[0] = l.at(1);
        t.m[0] = l.at(-1);
    }
    if (d2 < dim) {
        const Line l = line_of(q, z, d2);
        t.p[1] = l.at(1);
        t.m[1] = l.at(-1);
    }
    return t;
}

// a + coef (sum over the transverse pairs of b(+) + b(-) - 2 nt b(z)), the
// arithmetic of lap_combine_kernel
__device__ __forceinline__ double lap_t(const double* __restrict__ b, long long o, long long z, const Transverse& t,
                                        double a, double coef) {
    if (t.nt == 0) return a;
    double sn = b[o + t.p[0]] + b[o + t.m[0]];
    if (t.nt == 2) sn = sn + (b[o + t.p[1]] + b[o + t.m[1]]);
    return fma(coef, fma(-2.0 * t.nt, b[o + z], sn), a);
}

// Fc = HLLC between the face-centre states (WL, WR less L_t/24 of themselves,
// formed here from the transverse neighbours), F2 = HLLC between WL and WR;
// species: mass flux times X of the side upwind of the contact
template <int DIM>
__global__ void face_hllc4_kernel(int nspec, double g, double gm1_inv, int dir, long long N,
                                  const BoxDev* __restrict__ boxes, int nbox, const double* __restrict__ WL,
                                  const double* __restrict__ WR, double* __restrict__ Fc, double* __restrict__ F2) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    constexpr int NH = 2 + DIM;
    const int nv = NH + nspec;
    const ZoneCoord q = zone_coord(boxes, nbox, z);
    const Transverse t = transverse_of(q, z, DIM, dir);
    constexpr double c24 = -1.0 / 24.0;
    double qL[NH], qR[NH], Fh[NH];
    // face centres
#pragma unroll
    for (int f = 0; f < NH; f++) {
        const long long o = (long long)f * N;
        qL[f] = lap_t(WL, o, z, t, WL[o + z], c24);
        qR[f] = lap_t(WR, o, z, t, WR[o + z], c24);
    }
    double Ss = hllc_hydro<DIM>(g, gm1_inv, dir, qL, qR, Fh);
#pragma unroll
    for (int f = 0; f < NH; f++) Fc[(long long)f * N + z] = Fh[f];
    {
        const double* X = nonneg(Ss) ? WL : WR;
        for (int f = NH; f < nv; f++) {
            const long long o = (long long)f * N;
            Fc[o + z] = Fh[0] * lap_t(X, o, z, t, X[o + z], c24);
        }
    }
    // face averages
#pragma unroll
    for (int f = 0; f < NH; f++) {
        qL[f] = WL[(long long)f * N + z];
        qR[f] = WR[(long long)f * N + z];
    }
    Ss = hllc_hydro<DIM>(g, gm1_inv, dir, qL, qR, Fh);
#pragma unroll
    for (int f = 0; f < NH; f++) F2[(long long)f * N + z] = Fh[f];
    const double* X = nonneg(Ss) ? WL : WR;
    for (int f = NH; f < nv; f++) F2[(long long)f * N + z] = Fh[0] * X[(long long)f * N + z];
}

// A (first direction: =, else -=) the flux difference over dx
__global__ void div_kernel(int dir, int nf, long long N, const BoxDev* __restrict__ boxes, int nbox,
                           const double* __restrict__ Fa, double* __restrict__ A, int first) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const ZoneCoord q = zone_coord(boxes, nbox, z);
    const double idx = boxes[box_index(boxes, nbox, z)].idx[dir];
    const long long zm = line_of(q, z, dir).at(-1);
    for (int f = 0; f < nf; f++) {
        const long long o = (long long)f * N;
        const double d = (Fa[o + z] - Fa[o + zm]) * idx;
        A[o + z] = first ? -d : A[o + z] - d;
    }
}

// <R> = R_c + L R_c/24 (written), then <U> = <rhs> + dt_m <R> on the reactive
// fields and <rhs> on mass and momenta, in one pass
__global__ void lap_update4_kernel(int nvar, int dim, long long N, const BoxDev* __restrict__ boxes, int nbox,
                                   const double* __restrict__ Rc, const double* __restrict__ rhs,
                                   const double* __restrict__ dt_dev, double dt_frac, double dtm_host,
                                   double* __restrict__ R, double* __restrict__ U) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const LapNb nb = lap_nb(zone_coord(boxes, nbox, z), z, dim, -1);
    const double dtm = dt_dev ? (*dt_dev) * dt_frac : dtm_host;
    for (int f = 0; f < nvar; f++) {
        const long long i = (long long)f * N + z;
        double v = rhs[i];
        if (f >= 1 + dim) {
            const long long o = (long long)(f - 1 - dim) * N;
            const double r = lap_at(Rc, o, z, nb, Rc[o + z], 1.0 / 24.0);
            R[o + z] = r;
            v += dtm * r;
        }
        U[i] = v;
    }
}

cudaError_t lap(int dim, int nf, long long N, const BoxDev* boxes, int nbox, const double* a, const double* b,
                double coef, int skip, double* out, cudaStream_t st) {
    lap_combine_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(dim, nf, N, boxes, nbox, a, b, coef, skip, out);
    return cudaGetLastError();
}

cudaError_t launch_face_flux(const NetParams& P, int dim, int dir, long long N, const FourthWs& w, cudaStream_t st) {
    const double gi = 1.0 / P.gm1;
    switch (dim) {
        case 1: face_flux_kernel<1><<<fgrid(N), F_BLOCK, 0, st>>>(P.nspec, gi, dir, N, w.Wfc, w.Wf, w.Fc, w.F2); break;
        case 2: face_flux_kernel<2><<<fgrid(N), F_BLOCK, 0, st>>>(P.nspec, gi, dir, N, w.Wfc, w.Wf, w.Fc, w.F2); break;
        default: face_flux_kernel<3><<<fgrid(N), F_BLOCK, 0, st>>>(P.nspec, gi, dir, N, w.Wfc, w.Wf, w.Fc, w.F2); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_face_hllc4(const NetParams& P, int dim, int dir, long long N, const BoxDev* boxes, int nbox,
                              const FourthWs& w, cudaStream_t st) {
    const double g = P.gamma, gi = 1.0 / P.gm1;
    switch (dim) {
        case 1:
            face_hllc4_kernel<1><<<fgrid(N), F_BLOCK, 0, st>>>(P.nspec, g, gi, dir, N, boxes, nbox, w.WL, w.WR, w.Fc,
                                                                w.F2);
            break;
        case 2:
            face_hllc4_kernel<2><<<fgrid(N), F_BLOCK, 0, st>>>(P.nspec, g, gi, dir, N, boxes, nbox, w.WL, w.WR, w.Fc,
                                                                w.F2);
            break;
        default:
            face_hllc4_kernel<3><<<fgrid(N), F_BLOCK, 0, st>>>(P.nspec, g, gi, dir, N, boxes, nbox, w.WL, w.WR, w.Fc,
                                                                w.F2);
            break;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_advective4(const NetParams& P, int dim, int limiter, long long N, const BoxDev* boxes, int nbox,
                              const double* U, double* A, const FourthWs& w, cudaStream_t st) {
    const int nv = 2 + dim + P.nspec;
    cudaError_t e;
    prims4_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(dim, P.nspec, P.gm1, N, boxes, nbox, U, w.Wc, w.W2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = lap(dim, nv, N, boxes, nbox, w.Wc, w.W2, 1.0 / 24.0, -1, w.Wa, st)) != cudaSuccess) return e;
    for (int dir = 0; dir < dim; dir++) {
        if (limiter) {
            // face averages, face and zone limiters in one pass; HLLC with the
            // face-centre maps formed in place
            limit4_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(dim, P.nspec, dir, N, boxes, nbox, w.Wa, w.WL, w.WR);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = launch_face_hllc4(P, dim, dir, N, boxes, nbox, w, st)) != cudaSuccess) return e;
        } else {
            face_avg_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(dir, nv, N, boxes, nbox, w.Wa, w.Wf);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = lap(dim, nv, N, boxes, nbox, w.Wf, w.Wf, -1.0 / 24.0, dir, w.Wfc, st)) != cudaSuccess) return e;
            if ((e = launch_face_flux(P, dim, dir, N, w, st)) != cudaSuccess) return e;
        }
        // face-average fluxes once per face (fused into the divergence, each face's
        // map would be formed twice on the FP64 pipe), then the divergence
        if ((e = lap(dim, nv, N, boxes, nbox, w.Fc, w.F2, 1.0 / 24.0, dir, w.Fa, st)) != cudaSuccess) return e;
        div_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(dir, nv, N, boxes, nbox, w.Fa, A, dir == 0 ? 1 : 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_reaction_source4(const NetParams& P, int dim, long long N, const BoxDev* boxes, int nbox,
                                    const double* U, double* R, const FourthWs& w, cudaStream_t st) {
    const int nv = 2 + dim + P.nspec, n = P.nspec + 1;
    cudaError_t e;
    if ((e = lap(dim, nv, N, boxes, nbox, U, U, -1.0 / 24.0, -1, w.Uc, st)) != cudaSuccess) return e;
    if ((e = launch_reaction_source(P, N, dim, w.Uc, w.Rc, st)) != cudaSuccess) return e;
    return lap(dim, n, N, boxes, nbox, w.Rc, w.Rc, 1.0 / 24.0, -1, R, st);
}

cudaError_t launch_newton4(const NetParams& P, const NewtonCfg& cfg, int prec, int dim, long long N,
                           const BoxDev* boxes, int nbox, const double* rhs, const double* guess, double* Uout,
                           double* Rout, const double* dt_dev, double dt_frac, double dtm_host, int* zone_status,
                           int* zone_iters, DevStats* stats, const FourthWs& w, cudaStream_t st, int variant,
                           unsigned long long* queue, int persistent_blocks) {
    const int nv = 2 + dim + P.nspec, n = P.nspec + 1;
    cudaError_t e;
    lap_pair_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(dim, nv, N, boxes, nbox, rhs, w.rc, guess, w.gc, -1.0 / 24.0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_newton(P, cfg, prec, N, dim, w.rc, w.gc, nullptr, w.gc, w.Rc, dt_dev, dt_frac, dtm_host, zone_status,
                           zone_iters, stats, st, variant, queue, persistent_blocks)) != cudaSuccess)
        return e;
    (void)n;
    lap_update4_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(nv, dim, N, boxes, nbox, w.Rc, rhs, dt_dev, dt_frac, dtm_host,
                                                     Rout, Uout);
    return cudaGetLastError();
}

}  // namespace sdcd
