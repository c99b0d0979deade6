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
// the average, or of the averages at distance one or two, differences within
// 1e-12 of the averages counting as ties) and by the PPM
// overshoot bounds elsewhere; the limited mass fractions are renormalised; the
// two sides of a face then give its flux by HLLC, at the face centres and from
// the face averages alike.  The averaged source is R(U_c) + L R(U_c)/24; the implicit update is solved at
// zone centres (U_c - dt_m R(U_c) = rhs_c) and gives <U> = <rhs> + dt_m <R>.
// Every operator is a sequence of elementwise kernels over field-major arrays,
// one thread per zone, periodic within each box.  GB300 issues FP64 at 2 lanes
// per SM per clock, so even these stencils are bound by the FP64 pipe: the
// kernels divide once per zone (a Newton-Raphson reciprocal) and multiply.
#include "sdc_fourth_launch.h"
#include "sdc_launch.h"

namespace sdcd {
namespace {

constexpr int F_BLOCK = 256;
constexpr int F_MAXV = 2 + 3 + SDCD_MAXS;

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

// index of the zone o steps from q along d (periodic in the box)
__device__ __forceinline__ long long neighbour(const ZoneCoord& q, int d, int o) {
    int c[3] = {q.c[0], q.c[1], q.c[2]};
    c[d] = ((c[d] + o) % q.n[d] + q.n[d]) % q.n[d];
    return q.off + (long long)(c[0] + q.n[0] * (c[1] + q.n[1] * c[2]));
}

// out = a + coef * sum_{d < dim, d != skip} (b(z+e_d) - 2 b(z) + b(z-e_d)), nf fields,
// formed as a + coef (sum of the neighbour pairs - 2 n_d b(z)): per field one add
// per neighbour, then two FMAs (the FP64 pipe is the bound)
__global__ void lap_combine_kernel(int dim, int nf, long long N, const BoxDev* __restrict__ boxes, int nbox,
                                   const double* __restrict__ a, const double* __restrict__ b, double coef, int skip,
                                   double* __restrict__ out) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const ZoneCoord q = zone_coord(boxes, nbox, z);
    long long zp[3] = {z, z, z}, zm[3] = {z, z, z};
    int nd = 0;
    for (int d = 0; d < dim; d++) {
        zp[d] = neighbour(q, d, 1);
        zm[d] = neighbour(q, d, -1);
        if (d != skip) nd++;
    }
    const double c2 = -2.0 * nd;
    for (int f = 0; f < nf; f++) {
        const long long o = (long long)f * N;
        double sn = 0.0;
        bool first = true;
        for (int d = 0; d < dim; d++) {
            if (d == skip) continue;
            const double pair = b[o + zp[d]] + b[o + zm[d]];
            sn = first ? pair : sn + pair;
            first = false;
        }
        out[o + z] = fma(coef, fma(c2, b[o + z], sn), a[o + z]);
    }
}

// primitives (rho, u, p, X) of the conserved fields, field-major
__global__ void prim_kernel(int dim, int nspec, double gm1, long long N, const double* __restrict__ U,
                            double* __restrict__ W) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const double rho = U[z], ir = rcp_nr(rho);  // one reciprocal, then products (FP64 pipe)
    W[z] = rho;
    double ke = 0.0;
    for (int d = 0; d < dim; d++) {
        const double m = U[(1 + d) * N + z], u = m * ir;
        W[(1 + d) * N + z] = u;
        ke += 0.5 * m * u;
    }
    W[(1 + dim) * N + z] = gm1 * (U[(1 + dim) * N + z] - ke);
    for (int s = 0; s < nspec; s++) W[(2 + dim + s) * N + z] = U[(2 + dim + s) * N + z] * ir;
}

// face averages of the primitives, the face between z and its +1 neighbour along dir
__global__ void face_avg_kernel(int dir, int nf, long long N, const BoxDev* __restrict__ boxes, int nbox,
                                const double* __restrict__ Wa, double* __restrict__ Wf) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const ZoneCoord q = zone_coord(boxes, nbox, z);
    const long long zm = neighbour(q, dir, -1), zp = neighbour(q, dir, 1), zpp = neighbour(q, dir, 2);
    for (int f = 0; f < nf; f++) {
        const long long o = (long long)f * N;
        Wf[o + z] = 7.0 / 12.0 * (Wa[o + z] + Wa[o + zp]) - 1.0 / 12.0 * (Wa[o + zm] + Wa[o + zpp]);
    }
}

// physical Euler flux along dir of the primitive state q
__device__ __forceinline__ void euler_flux(int dim, int nspec, double igm1, int dir, const double* q, double* F) {
    const double rho = q[0], un = q[1 + dir], p = q[1 + dim];
    double k2 = 0.0;
    for (int d = 0; d < dim; d++) k2 = fma(q[1 + d], q[1 + d], k2);
    const double E = fma(p, igm1, 0.5 * rho * k2);
    F[0] = rho * un;
    for (int d = 0; d < dim; d++) F[1 + d] = rho * un * q[1 + d] + (d == dir ? p : 0.0);
    F[1 + dim] = (E + p) * un;
    for (int s = 0; s < nspec; s++) F[2 + dim + s] = rho * un * q[2 + dim + s];
}

// Fc = F(Wfc) (face centres), F2 = F(Wf) (from the face averages)
__global__ void face_flux_kernel(int dim, int nspec, double igm1, int dir, long long N,
                                 const double* __restrict__ Wfc, const double* __restrict__ Wf,
                                 double* __restrict__ Fc, double* __restrict__ F2) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const int nv = 2 + dim + nspec;
    double q[F_MAXV], F[F_MAXV];
    for (int f = 0; f < nv; f++) q[f] = Wfc[(long long)f * N + z];
    euler_flux(dim, nspec, igm1, dir, q, F);
    for (int f = 0; f < nv; f++) Fc[(long long)f * N + z] = F[f];
    for (int f = 0; f < nv; f++) q[f] = Wf[(long long)f * N + z];
    euler_flux(dim, nspec, igm1, dir, q, F);
    for (int f = 0; f < nv; f++) F2[(long long)f * N + z] = F[f];
}

// ---- limited form
constexpr double CS_C = 1.25;  // bound of the limited curvature over its neighbours'

__device__ __forceinline__ bool same_sign3(double a, double b, double c) {
    return (a > 0.0 && b > 0.0 && c > 0.0) || (a < 0.0 && b < 0.0 && c < 0.0);
}

// face between zones a0 and ap (neighbours am, app): a value outside [a0, ap]
// becomes (a0 + ap)/2 - d2/6, d2 the second difference 3 (a0 - 2 af + ap)
// limited by C times those of the two zones; the unlimited d2 returns af itself
__device__ __forceinline__ double cs_face(double am, double a0, double ap, double app, double af) {
    if ((af - a0) * (ap - af) < 0.0) {
        const double d2f = 3.0 * (a0 - 2.0 * af + ap);
        const double d2l = am - 2.0 * a0 + ap, d2r = a0 - 2.0 * ap + app;
        double d2 = 0.0;
        if (same_sign3(d2f, d2l, d2r)) {
            const double m = fmin(fmin(CS_C * fabs(d2l), CS_C * fabs(d2r)), fabs(d2f));
            d2 = d2f > 0.0 ? m : -m;
        }
        af = 0.5 * (a0 + ap) - d2 * (1.0 / 6.0);
    }
    return af;
}

// a difference of two averages, zero within 1e-12 of their magnitudes:
// averages mirrored across a plane of symmetry of the data differ only by
// rounding, and the extremum tests would take their branch from its order
constexpr double CS_FLAT = 1e-12;
__device__ __forceinline__ double avg_diff(double a, double b) {
    const double d = a - b;
    return fabs(d) <= CS_FLAT * (fabs(a) + fabs(b)) ? 0.0 : d;
}

// zone a0 (neighbours amm .. app) with face values fm (lower) and fp (upper)
__device__ __forceinline__ void cs_zone(double amm, double am, double a0, double ap, double app, double& fm,
                                        double& fp) {
    const double dm = fm - a0, dp = fp - a0;
    if (dp * dm >= 0.0 || avg_diff(am, a0) * avg_diff(a0, ap) <= 0.0 ||
        avg_diff(amm, a0) * avg_diff(a0, app) <= 0.0) {
        // extremum: scale both deviations by the limited curvature over the parabola's
        const double d2 = 6.0 * (fm + fp - 2.0 * a0);
        const double d2c = am - 2.0 * a0 + ap, d2l = amm - 2.0 * am + a0, d2r = a0 - 2.0 * ap + app;
        double lim = 0.0;
        if (same_sign3(d2, d2c, d2l) && same_sign3(d2, d2c, d2r)) {
            const double m = fmin(fmin(fabs(d2), CS_C * fabs(d2c)), fmin(CS_C * fabs(d2l), CS_C * fabs(d2r)));
            lim = d2 > 0.0 ? m : -m;
        }
        const double s = d2 != 0.0 ? lim / d2 : 0.0;
        fm = fma(dm, s, a0);
        fp = fma(dp, s, a0);
    } else {
        // monotone: the parabola may not overshoot the far face
        if (fabs(dp) >= 2.0 * fabs(dm)) fp = a0 - 2.0 * dm;
        if (fabs(dm) >= 2.0 * fabs(dp)) fm = a0 - 2.0 * dp;
    }
}

// Wl = face-limited face averages (the face between z and its +1 neighbour along dir)
__global__ void limit_face_kernel(int dir, int nf, long long N, const BoxDev* __restrict__ boxes, int nbox,
                                  const double* __restrict__ Wa, const double* __restrict__ Wf,
                                  double* __restrict__ Wl) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const ZoneCoord q = zone_coord(boxes, nbox, z);
    const long long zm = neighbour(q, dir, -1), zp = neighbour(q, dir, 1), zpp = neighbour(q, dir, 2);
    for (int f = 0; f < nf; f++) {
        const long long o = (long long)f * N;
        Wl[o + z] = cs_face(Wa[o + zm], Wa[o + z], Wa[o + zp], Wa[o + zpp], Wf[o + z]);
    }
}

// zone z limits its two face values: WL[z] = its upper face (left side of the
// face z+1/2), WR[z-1] = its lower face (right side of the face z-1/2)
__global__ void limit_zone_kernel(int dim, int nspec, int dir, long long N, const BoxDev* __restrict__ boxes,
                                  int nbox, const double* __restrict__ Wa, const double* __restrict__ Wl,
                                  double* __restrict__ WL, double* __restrict__ WR) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const ZoneCoord q = zone_coord(boxes, nbox, z);
    const long long zmm = neighbour(q, dir, -2), zm = neighbour(q, dir, -1);
    const long long zp = neighbour(q, dir, 1), zpp = neighbour(q, dir, 2);
    const int nh = 2 + dim, nv = nh + nspec;
    double fm[F_MAXV], fp[F_MAXV];
    for (int f = 0; f < nv; f++) {
        const long long o = (long long)f * N;
        fm[f] = Wl[o + zm];
        fp[f] = Wl[o + z];
        cs_zone(Wa[o + zmm], Wa[o + zm], Wa[o + z], Wa[o + zp], Wa[o + zpp], fm[f], fp[f]);
    }
    if (nspec > 0) {
        double sm = 0.0, sp = 0.0;
        for (int s = 0; s < nspec; s++) {
            sm += fm[nh + s];
            sp += fp[nh + s];
        }
        for (int s = 0; s < nspec; s++) {
            fm[nh + s] /= sm;
            fp[nh + s] /= sp;
        }
    }
    for (int f = 0; f < nv; f++) {
        WL[(long long)f * N + z] = fp[f];
        WR[(long long)f * N + zm] = fm[f];
    }
}

// Fc = HLLC(WLc, WRc) (face centres), F2 = HLLC(WL, WR) (from the face
// averages); species: mass flux times X of the side upwind of the contact
template <int DIM>
__global__ void face_hllc_kernel(int nspec, double g, double gm1_inv, int dir, long long N,
                                 const double* __restrict__ WLc, const double* __restrict__ WRc,
                                 const double* __restrict__ WL, const double* __restrict__ WR,
                                 double* __restrict__ Fc, double* __restrict__ F2) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    constexpr int NH = 2 + DIM;
    const int nv = NH + nspec;
    for (int side = 0; side < 2; side++) {
        const double* L = side ? WL : WLc;
        const double* R = side ? WR : WRc;
        double* F = side ? F2 : Fc;
        double qL[NH], qR[NH], Fh[NH];
#pragma unroll
        for (int f = 0; f < NH; f++) {
            qL[f] = L[(long long)f * N + z];
            qR[f] = R[(long long)f * N + z];
        }
        const double Ss = hllc_hydro<DIM>(g, gm1_inv, dir, qL, qR, Fh);
#pragma unroll
        for (int f = 0; f < NH; f++) F[(long long)f * N + z] = Fh[f];
        const double* Xup = Ss >= 0.0 ? L : R;
        for (int f = NH; f < nv; f++) F[(long long)f * N + z] = Fh[0] * Xup[(long long)f * N + z];
    }
}

// A (first direction: =, else -=) the flux difference over dx
__global__ void div_kernel(int dir, int nf, long long N, const BoxDev* __restrict__ boxes, int nbox,
                           const double* __restrict__ Fa, double* __restrict__ A, int first) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const ZoneCoord q = zone_coord(boxes, nbox, z);
    const double idx = boxes[box_index(boxes, nbox, z)].idx[dir];
    const long long zm = neighbour(q, dir, -1);
    for (int f = 0; f < nf; f++) {
        const long long o = (long long)f * N;
        const double d = (Fa[o + z] - Fa[o + zm]) * idx;
        A[o + z] = first ? -d : A[o + z] - d;
    }
}

// <U> = <rhs> + dt_m <R> on the reactive fields, <rhs> on mass and momenta
__global__ void update4_kernel(int nvar, int dim, long long N, const double* __restrict__ rhs,
                               const double* __restrict__ R, const double* __restrict__ dt_dev, double dt_frac,
                               double dtm_host, double* __restrict__ U) {
    // one thread per zone, every field (no 64-bit division per element)
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const double dtm = dt_dev ? (*dt_dev) * dt_frac : dtm_host;
    for (int f = 0; f < nvar; f++) {
        const long long i = (long long)f * N + z;
        double v = rhs[i];
        if (f >= 1 + dim) v += dtm * R[(long long)(f - 1 - dim) * N + z];
        U[i] = v;
    }
}

cudaError_t lap(int dim, int nf, long long N, const BoxDev* boxes, int nbox, const double* a, const double* b,
                double coef, int skip, double* out, cudaStream_t st) {
    lap_combine_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(dim, nf, N, boxes, nbox, a, b, coef, skip, out);
    return cudaGetLastError();
}

cudaError_t launch_face_hllc(const NetParams& P, int dim, int dir, long long N, const FourthWs& w, cudaStream_t st) {
    const double g = P.gamma, gi = 1.0 / P.gm1;
    switch (dim) {
        case 1:
            face_hllc_kernel<1><<<fgrid(N), F_BLOCK, 0, st>>>(P.nspec, g, gi, dir, N, w.WLc, w.WRc, w.WL, w.WR, w.Fc,
                                                               w.F2);
            break;
        case 2:
            face_hllc_kernel<2><<<fgrid(N), F_BLOCK, 0, st>>>(P.nspec, g, gi, dir, N, w.WLc, w.WRc, w.WL, w.WR, w.Fc,
                                                               w.F2);
            break;
        default:
            face_hllc_kernel<3><<<fgrid(N), F_BLOCK, 0, st>>>(P.nspec, g, gi, dir, N, w.WLc, w.WRc, w.WL, w.WR, w.Fc,
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
    if ((e = lap(dim, nv, N, boxes, nbox, U, U, -1.0 / 24.0, -1, w.Uc, st)) != cudaSuccess) return e;
    prim_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(dim, P.nspec, P.gm1, N, U, w.W2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    prim_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(dim, P.nspec, P.gm1, N, w.Uc, w.Wc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = lap(dim, nv, N, boxes, nbox, w.Wc, w.W2, 1.0 / 24.0, -1, w.Wa, st)) != cudaSuccess) return e;
    for (int dir = 0; dir < dim; dir++) {
        face_avg_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(dir, nv, N, boxes, nbox, w.Wa, w.Wf);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (limiter) {
            // Wfc holds the face-limited averages here
            limit_face_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(dir, nv, N, boxes, nbox, w.Wa, w.Wf, w.Wfc);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            limit_zone_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(dim, P.nspec, dir, N, boxes, nbox, w.Wa, w.Wfc, w.WL,
                                                            w.WR);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = lap(dim, nv, N, boxes, nbox, w.WL, w.WL, -1.0 / 24.0, dir, w.WLc, st)) != cudaSuccess) return e;
            if ((e = lap(dim, nv, N, boxes, nbox, w.WR, w.WR, -1.0 / 24.0, dir, w.WRc, st)) != cudaSuccess) return e;
            if ((e = launch_face_hllc(P, dim, dir, N, w, st)) != cudaSuccess) return e;
        } else {
            if ((e = lap(dim, nv, N, boxes, nbox, w.Wf, w.Wf, -1.0 / 24.0, dir, w.Wfc, st)) != cudaSuccess) return e;
            face_flux_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(dim, P.nspec, 1.0 / P.gm1, dir, N, w.Wfc, w.Wf, w.Fc,
                                                           w.F2);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
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
    if ((e = lap(dim, nv, N, boxes, nbox, rhs, rhs, -1.0 / 24.0, -1, w.rc, st)) != cudaSuccess) return e;
    if ((e = lap(dim, nv, N, boxes, nbox, guess, guess, -1.0 / 24.0, -1, w.gc, st)) != cudaSuccess) return e;
    if ((e = launch_newton(P, cfg, prec, N, dim, w.rc, w.gc, w.gc, w.Rc, dt_dev, dt_frac, dtm_host, zone_status,
                           zone_iters, stats, st, variant, queue, persistent_blocks)) != cudaSuccess)
        return e;
    if ((e = lap(dim, n, N, boxes, nbox, w.Rc, w.Rc, 1.0 / 24.0, -1, Rout, st)) != cudaSuccess) return e;
    update4_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(nv, dim, N, rhs, Rout, dt_dev, dt_frac, dtm_host,
                                                                  Uout);
    return cudaGetLastError();
}

}  // namespace sdcd
