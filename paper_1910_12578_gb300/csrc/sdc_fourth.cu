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
// The averaged source is R(U_c) + L R(U_c)/24; the implicit update is solved at
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

}  // namespace

cudaError_t launch_advective4(const NetParams& P, int dim, long long N, const BoxDev* boxes, int nbox,
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
        if ((e = lap(dim, nv, N, boxes, nbox, w.Wf, w.Wf, -1.0 / 24.0, dir, w.Wfc, st)) != cudaSuccess) return e;
        face_flux_kernel<<<fgrid(N), F_BLOCK, 0, st>>>(dim, P.nspec, 1.0 / P.gm1, dir, N, w.Wfc, w.Wf, w.Fc, w.F2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
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
