// sdc_stencil_split.cuh -- the advective term A(U) of Eq. 1 (paper section 2)
// in three direction passes, the last one fused with the right-hand side of
// Eq. sdc:general.
//
// The arithmetic per zone and per face is that of stencil_kernel (the same
// primitives, MC half slopes, HLLC, upwind renormalised species flux and flux
// difference, accumulated over x, y, z in that order), so the results agree
// with it bit for bit.  What differs is how the work is laid out: on GB300 the
// stencil is bound by the narrow FP64 pipe, not by HBM, so this form trades
// bandwidth for arithmetic.  Each pass stages lines of zones along its own
// direction only, with a 2-zone halo along that direction and none across it,
// so every zone's primitives are formed once (the x pass, which also writes
// them to a field-major buffer for the y and z passes), every one-sided
// difference once per face, every half slope once per zone and every face
// flux once, apart from the halo of the line ends.  The passes hand the
// partial sum of A to each other through global memory (a few hundred bytes
// per zone, against the hundreds of FP64 operations per zone that a 3D tile's
// halo recomputes).
//
// A CTA owns NL lines of L zones along direction D (x: 8 lines of 32; y, z:
// 16 lines of 16, the lines adjacent along x so that loads and stores
// coalesce).  Phases, one work item per thread in each:
//   1. stage the primitives of the L + 4 zones of every line (periodic wrap
//      inside the box);
//   2. one-sided differences of neighbouring zones, L + 3 per line;
//   3. half slopes from the two differences of a zone, L + 2 per line;
//   4. face fluxes, L + 1 per line (for the species the upwind X_s and the
//      factor F_rho / (sum X) / dx_D, so that phase 5 takes each species'
//      flux difference in two fused multiply-adds);
//   5. A += -(F_{i+1/2} - F_{i-1/2}) / dx_D for the L zones of every line.
#pragma once
#include "sdc_stencil.cuh"

namespace sdcd {

__device__ __forceinline__ void prefetch_l2(const double* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

template <int D> struct SplitShape;
template <> struct SplitShape<0> { static constexpr int L = 32, NL = 8; };
template <> struct SplitShape<1> { static constexpr int L = 16, NL = 16; };
template <> struct SplitShape<2> { static constexpr int L = 16, NL = 16; };

template <int D>
struct SplitGeom {
    static constexpr int L = SplitShape<D>::L, NL = SplitShape<D>::NL;
    static constexpr int NQ = NL * (L + 4);   // staged zones
    static constexpr int ND = NL * (L + 3);   // one-sided differences
    static constexpr int NH = NL * (L + 2);   // half slopes
    static constexpr int NF = NL * (L + 1);   // faces
    static constexpr int NO = NL * L;         // zones written
    static constexpr int THREADS = NQ;        // >= every phase's work items
    static constexpr int NB = ND;             // second buffer: differences, then half slopes
    // the line axis (across the lines) and the axis held fixed by a tile
    static constexpr int A = D == 0 ? 1 : 0;
    static constexpr int T = D == 2 ? 1 : 2;
    // work item i of a phase with n positions per line -> (line, position):
    // x lines position-fastest (the x zones of a line are contiguous), y and
    // z lines line-fastest (neighbouring lines are neighbouring x columns)
    __device__ static __forceinline__ void item(int i, int n, int& li, int& j) {
        if (D == 0) { li = i / n; j = i - li * n; }
        else { j = i / NL; li = i - j * NL; }
    }
    // shared-memory slot of (line, position) in an array of n positions per line
    __device__ static __forceinline__ int slot(int li, int j, int n) { return D == 0 ? li * n + j : j * NL + li; }
};

template <int NS, int D>
constexpr size_t split_smem_bytes() {
    using G = SplitGeom<D>;
    return sizeof(double) * (size_t)(5 + NS) * (G::NQ + G::NB);
}

// CTAs per SM requested by the launch bounds: two where both fit in shared memory
template <int NS, int D>
constexpr int split_min_blocks() {
    return 2 * split_smem_bytes<NS, D>() <= 220 * 1024 ? 2 : 1;
}

// FIRST: the pass that reads the conserved state U and writes the primitives
// to prim; the others read prim.  LAST: the pass that finishes A (and, for
// MODE == STENCIL_A_RHS, forms the rhs); the others leave partial sums in A.
template <int NS, int D, bool FIRST, bool LAST, int MODE>
__global__ void __launch_bounds__(SplitGeom<D>::THREADS, split_min_blocks<NS, D>())
stencil_split_kernel(NetParams P, int limiter, long long Ntot, const BoxDev* __restrict__ boxes,
                     const TileDev* __restrict__ tiles, const double* __restrict__ U, double* __restrict__ prim,
                     double* __restrict__ Aout, RhsArgs ra) {
    constexpr int DIM = 3;
    using G = SplitGeom<D>;
    constexpr int L = G::L, NL = G::NL;
    constexpr int NV = 2 + DIM + NS;
    constexpr int NHY = 2 + DIM;  // hydrodynamic fields
    extern __shared__ double smem[];
    double* sq = smem;                // [NV][NQ] primitives, then face fluxes
    double* sb = smem + NV * G::NQ;   // [NV][NB] differences, then half slopes

    const TileDev t = tiles[blockIdx.x];
    const BoxDev b = boxes[t.box];
    const int tid = threadIdx.x;
    const int nD = b.n[D], nA = b.n[G::A];
    const double gm1 = P.gm1;

    // global zone index of (line, position p along D relative to the tile origin)
    auto zone_of = [&](int li, int p) -> long long {
        int c[3];
        c[D] = wrap(t.o[D] + p, nD);
        c[G::A] = t.o[G::A] + li;
        c[G::T] = t.o[G::T];
        return b.off + c[0] + (long long)b.n[0] * (c[1] + (long long)b.n[1] * c[2]);
    };

    // the global data of phase 5 (the partial sums of A, and with the rhs the
    // node state, the previous iterate's A and R), requested into L2 now so
    // that the end of the tile does not wait on HBM
    if (!FIRST && tid < G::NO) {
        int li, p;
        G::item(tid, L, li, p);
        if (t.o[G::A] + li < nA && t.o[D] + p < nD) {
            const long long gi = zone_of(li, p);
#pragma unroll
            for (int f = 0; f < NV; f++) prefetch_l2(Aout + f * Ntot + gi);
            if (LAST && MODE == STENCIL_A_RHS) {
#pragma unroll
                for (int f = 0; f < NV; f++) {
                    prefetch_l2(U + f * Ntot + gi);
                    prefetch_l2(ra.Aold_m + f * Ntot + gi);
                }
#pragma unroll
                for (int r = 0; r < NV - 1 - DIM; r++) prefetch_l2(ra.Rnext + r * Ntot + gi);
            }
        }
    }
    // ---- 1. stage the primitives of every line and its halo
    {
        int li, j;
        G::item(tid, L + 4, li, j);
        if (tid < G::NQ && t.o[G::A] + li < nA) {
            const long long gi = zone_of(li, j - 2);
            const int s = G::slot(li, j, L + 4);
            if (FIRST) {
                const double rho = __ldg(U + gi);
                const double ir = rcp_nr(rho);
                double ke = 0.0;
                double q[NV];
                q[0] = rho;
#pragma unroll
                for (int d = 0; d < DIM; d++) {
                    const double m = __ldg(U + (1 + d) * Ntot + gi);
                    const double u = m * ir;
                    q[1 + d] = u;
                    ke = fma(m, u, ke);
                }
                q[1 + DIM] = gm1 * fma(-0.5, ke, __ldg(U + (1 + DIM) * Ntot + gi));
#pragma unroll
                for (int sp = 0; sp < NS; sp++) q[2 + DIM + sp] = __ldg(U + (2 + DIM + sp) * Ntot + gi) * ir;
                // a zone of this tile (not a halo copy of another tile's) goes to the buffer
                const bool own = j >= 2 && j < L + 2 && t.o[D] + j - 2 < nD;
#pragma unroll
                for (int f = 0; f < NV; f++) {
                    sq[f * G::NQ + s] = q[f];
                    if (own) prim[f * Ntot + gi] = q[f];
                }
            } else {
#pragma unroll
                for (int f = 0; f < NV; f++) sq[f * G::NQ + s] = prim[f * Ntot + gi];
            }
        }
    }
    __syncthreads();
    // ---- 2. one-sided differences: d_j = q_{j+1} - q_j of staged positions j, j+1
    if (tid < G::ND) {
        int li, j;
        G::item(tid, L + 3, li, j);
        if (t.o[G::A] + li < nA) {
        const int s0 = G::slot(li, j, L + 4), s1 = G::slot(li, j + 1, L + 4), sd = G::slot(li, j, L + 3);
#pragma unroll
        for (int f = 0; f < NV; f++) sb[f * G::NB + sd] = sq[f * G::NQ + s1] - sq[f * G::NQ + s0];
        }
    }
    __syncthreads();
    // ---- 3. half slopes of the zones at positions -1..L (staged k + 1, k = 0..L+1)
    {
        double h[NV];
        int li = 0, k = 0;
        if (tid < G::NH) G::item(tid, L + 2, li, k);
        const bool act = tid < G::NH && t.o[G::A] + li < nA;
        if (act) {
            const int sl = G::slot(li, k, L + 3), sr = G::slot(li, k + 1, L + 3);
#pragma unroll
            for (int f = 0; f < NV; f++) h[f] = mc_half_slope_d(limiter, sb[f * G::NB + sl], sb[f * G::NB + sr]);
        }
        __syncthreads();  // every difference is read: the buffer takes the half slopes
        if (act) {
            const int sh = G::slot(li, k, L + 2);
#pragma unroll
            for (int f = 0; f < NV; f++) sb[f * G::NB + sh] = h[f];
        }
    }
    __syncthreads();
    // ---- 4. face fluxes: face m (m = 0..L) between zone positions m-1 and m
    {
        double F[NV];
        double fmi = 0.0;
        int li = 0, m = 0;
        if (tid < G::NF) G::item(tid, L + 1, li, m);
        const bool act = tid < G::NF && t.o[G::A] + li < nA;
        if (act) {
            const int zl = G::slot(li, m + 1, L + 4), zr = G::slot(li, m + 2, L + 4);
            const int hl = G::slot(li, m, L + 2), hr = G::slot(li, m + 1, L + 2);
            double qL[NHY], qR[NHY];
#pragma unroll
            for (int f = 0; f < NHY; f++) {
                qL[f] = sq[f * G::NQ + zl] + sb[f * G::NB + hl];
                qR[f] = sq[f * G::NQ + zr] - sb[f * G::NB + hr];
            }
            const double Ss = hllc_hydro<DIM>(P.gamma, P.gm1_inv, D, qL, qR, F);
            // species: the side upwind of the contact, renormalised
            const bool lft = nonneg(Ss);
            const int zu = lft ? zl : zr, hu = lft ? hl : hr;
            const long long flip = lft ? 0ll : SIGN_BIT;
            double X[NS];
            double sum = 0.0;
#pragma unroll
            for (int s = 0; s < NS; s++) {
                const double q = sq[(NHY + s) * G::NQ + zu], hh = sb[(NHY + s) * G::NB + hu];
                X[s] = q + bitsd(dbits(hh) ^ flip);
                sum += X[s];
            }
            // the face keeps X_s and fm / dx (fm = F_rho / sum X), as stencil_kernel
            fmi = F[0] * rcp_nr(sum) * b.idx[D];
#pragma unroll
            for (int s = 0; s < NS; s++) F[NHY + s] = X[s];
        }
        __syncthreads();  // every primitive and slope is read: the first buffer takes the fluxes
        if (act) {
            const int sf = G::slot(li, m, L + 1);
#pragma unroll
            for (int f = 0; f < NV; f++) sq[f * G::NQ + sf] = F[f];
            sb[sf] = fmi;
        }
    }
    __syncthreads();
    // ---- 5. flux difference of the zones of the tile
    if (tid >= G::NO) return;
    int li, p;
    G::item(tid, L, li, p);
    if (t.o[G::A] + li >= nA || t.o[D] + p >= nD) return;
    const long long gi = zone_of(li, p);
    const int flo = G::slot(li, p, L + 1), fhi = G::slot(li, p + 1, L + 1);
    const double idx = b.idx[D];
    double A[NV];
#pragma unroll
    for (int f = 0; f < NHY; f++) {
        const double prev = FIRST ? 0.0 : Aout[f * Ntot + gi];
        A[f] = fma(-(sq[f * G::NQ + fhi] - sq[f * G::NQ + flo]), idx, prev);
        Aout[f * Ntot + gi] = A[f];
    }
    // species: fm_lo X_lo / dx - fm_hi X_hi / dx, as stencil_kernel
    const double ml = sb[flo], mh = sb[fhi];
#pragma unroll
    for (int s = 0; s < NS; s++) {
        const int f = NHY + s;
        const double prev = FIRST ? 0.0 : Aout[f * Ntot + gi];
        A[f] = fma(-mh, sq[f * G::NQ + fhi], fma(ml, sq[f * G::NQ + flo], prev));
        Aout[f * Ntot + gi] = A[f];
    }
    if (LAST && MODE == STENCIL_A_RHS) {
        const double dt = *ra.dt;
        const double dtm = dt * ra.dtm_frac;
        double qdt[MAXM];
#pragma unroll
        for (int l = 0; l < MAXM; l++) qdt[l] = ra.qw[l] * dt;
#pragma unroll
        for (int f = 0; f < NV; f++) {
            double v = fma(dtm, A[f] - __ldg(ra.Aold_m + f * Ntot + gi), __ldg(U + f * Ntot + gi));
            const bool reactive = f >= 1 + DIM;
            const int r = f - 1 - DIM;
            if (reactive) v = fma(-dtm, __ldg(ra.Rnext + r * Ntot + gi), v);
            double I = 0.0;
#pragma unroll
            for (int l = 0; l < MAXM; l++) {
                if (l < ra.M) {
                    double src = __ldg(ra.Aold[l] + f * Ntot + gi);
                    if (reactive) src += __ldg(ra.Rold[l] + r * Ntot + gi);
                    I = fma(qdt[l], src, I);
                }
            }
            ra.rhs[f * Ntot + gi] = v + I;
        }
    }
}

}  // namespace sdcd
