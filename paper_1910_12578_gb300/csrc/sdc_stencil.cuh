// sdc_stencil.cuh -- advective term A(U) (paper section 2, Eq. 1: minus the
// divergence of the advective fluxes) fused with the right-hand side of the
// implicit update of Eq. sdc:general.
//
// Method of lines: conserved -> primitive (rho, u, p, X), per direction a
// piecewise-linear reconstruction with MC-limited (or unlimited centred)
// slopes, the upwind interface mass fractions renormalised to sum to one,
// HLLC flux (Davis wave speeds, species flux = X of the side upwind of the
// contact times the mass flux), A = -sum_d (F_{i+1/2} - F_{i-1/2}) / dx_d.
//
// One CTA owns a TX x TY x TZ tile of one box.  The primitives of the tile and
// of its 2-zone halo along each axis (a cross-shaped region; every box is
// periodic on itself, so the halo wraps inside the box) are staged once in
// shared memory.  Per direction: every zone's half slope is computed once into
// a shared buffer, every face flux once (one face per thread when the tile is
// a cube), the fluxes reuse the slope buffer, and each thread accumulates the
// flux difference of its zones.  GB300 runs FP64 at 1/61 of its FP32 rate,
// so divisions and square roots are refinements of hardware approximations and the limiter works on bit patterns (sdc_fastmath.cuh).
#pragma once
#include "sdc_dev.cuh"
#include "sdc_fastmath.cuh"

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
    const double* Aold[MAXM];  // A^{(k)} of the integral's terms
    const double* Rold[MAXM];  // R^{(k)} of the integral's terms ([n][Ntot])
    const double* Rnext;       // R^{m+1,(k)}
    const double* Aold_m;      // A^{m,(k)}
    double* rhs;
    const double* dt;          // device scalar: the step size
    double qw[MAXM];           // weights of the terms (units of dt)
    double dtm_frac;           // dt_m / dt
    int M;                     // number of terms
};

template <int DIM, int TX, int TY, int TZ>
struct TileGeom {
    static constexpr int HX = TX + 4;
    static constexpr int NXE = HX * TY * TZ;                 // x-extended slab
    static constexpr int NYH = (DIM >= 2) ? TX * 4 * TZ : 0;  // y halo slabs
    static constexpr int NZH = (DIM >= 3) ? TX * TY * 4 : 0;  // z halo slabs
    static constexpr int NC = NXE + NYH + NZH;
    // slopes: positions -1..T_d along d, the others inside the tile
    static constexpr int SX = (TX + 2) * TY * TZ;
    static constexpr int SY = (DIM >= 2) ? TX * (TY + 2) * TZ : 0;
    static constexpr int SZ = (DIM >= 3) ? TX * TY * (TZ + 2) : 0;
    static constexpr int NSL = SX > SY ? (SX > SZ ? SX : SZ) : (SY > SZ ? SY : SZ);
    static constexpr int FX = (TX + 1) * TY * TZ;
    static constexpr int FY = (DIM >= 2) ? TX * (TY + 1) * TZ : 0;
    static constexpr int FZ = (DIM >= 3) ? TX * TY * (TZ + 1) : 0;
    static constexpr int NF = FX > FY ? (FX > FZ ? FX : FZ) : (FY > FZ ? FY : FZ);
    static constexpr int NB = NSL > NF ? NSL : NF;           // slope / flux buffer
    static constexpr int NT = TX * TY * TZ;
    static constexpr int THREADS = NF;                       // one face per thread per direction
};

// CTAs per SM the launch bounds ask for: two where two tiles' shared memory
// (primitives, the slope / flux buffer and the per-face species flux factor)
// fit in an SM's 228 KB, so that one
// CTA's barrier phases overlap the other's arithmetic; the registers per
// thread are then capped at 64K / (2 THREADS).
template <int DIM, int NS, int TX, int TY, int TZ>
constexpr int stencil_min_blocks() {
    using G = TileGeom<DIM, TX, TY, TZ>;
    return sizeof(double) * ((size_t)(2 + DIM + NS) * (G::NC + G::NB) + G::NB) <= 112 * 1024 ? 2 : 1;
}

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

// HLLC flux of the hydrodynamic fields through a face normal to `dir`;
// q = [rho, u_0.., p].  Returns S* (its sign picks the species' upwind side).
// The sound speeds are gamma p / sqrt(gamma p rho) (no reciprocal of rho), the
// total energy is formed for the upwind side only, and the star state's energy
// flux uses fac * e* = (E (S - u) + (S* - u)(S* rho (S - u) + p)) / (S - S*),
// the same quantity as rho*_K E*_K with e* = E/rho + (S* - u)(S* + p/(rho (S - u))).
// Sign tests and the wave-speed min / max on bit patterns (integer pipe; FP64
// compares, min and max issue on the narrow FP64 pipe).  x >= 0 holds for +0
// and -0 as in IEEE; the min / max order -0 below +0 (IEEE leaves the pick
// between equal zeros open; the value is the same).
__device__ __forceinline__ bool nonneg(double x) { return dbits(x) >= 0 || mag2(x) == 0ull; }
__device__ __forceinline__ bool positive(double x) { return dbits(x) > 0; }
__device__ __forceinline__ long long ord_bits(double x) {
    const long long b = dbits(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}
__device__ __forceinline__ double min_d(double a, double b) { return ord_bits(a) <= ord_bits(b) ? a : b; }
__device__ __forceinline__ double max_d(double a, double b) { return ord_bits(a) >= ord_bits(b) ? a : b; }

template <int DIM>
__device__ __forceinline__ double hllc_hydro(double g, double gm1_inv, int dir, const double* qL, const double* qR,
                                             double* Fh) {
    const double rL = qL[0], rR = qR[0];
    const double unL = qL[1 + dir], unR = qR[1 + dir];
    const double pL = qL[1 + DIM], pR = qR[1 + DIM];
    const double gpL = g * pL, gpR = g * pR;
    const double cL = gpL * rsqrt_nr(gpL * rL), cR = gpR * rsqrt_nr(gpR * rR);
    const double SL = min_d(unL - cL, unR - cR);
    const double SR = max_d(unL + cL, unR + cR);
    const double dL = SL - unL, dR = SR - unR;
    const double aL = rL * dL, aR = rR * dR;  // mass fluxes relative to the waves
    const double Ss = (pR - pL + unL * aL - unR * aR) * rcp_nr(aL - aR);
    // region: SL >= 0 -> F_L; else Ss >= 0 -> F*_L; else SR > 0 -> F*_R; else F_R
    const bool left = nonneg(SL) || nonneg(Ss);
    const bool star = !nonneg(SL) && (nonneg(Ss) || positive(SR));
    const double r = left ? rL : rR, un = left ? unL : unR, p = left ? pL : pR;
    const double S = left ? SL : SR, a = left ? aL : aR, dS = left ? dL : dR;
    const double* q = left ? qL : qR;
    double k2 = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; d++) k2 = fma(q[1 + d], q[1 + d], k2);
    const double E = fma(p, gm1_inv, 0.5 * r * k2);
    Fh[0] = r * un;
#pragma unroll
    for (int d = 0; d < DIM; d++) Fh[1 + d] = r * un * q[1 + d] + (d == dir ? p : 0.0);
    Fh[1 + DIM] = (E + p) * un;
    if (star) {
        // U*_K = fac [1, S* (normal) / u_t, e*], fac = rho (S - u)/(S - S*)
        const double inv = rcp_nr(S - Ss);
        const double fac = a * inv;
        const double feS = fma(Ss - un, fma(Ss, a, p), E * dS) * inv;
        Fh[0] = fma(S, fac - r, Fh[0]);
#pragma unroll
        for (int d = 0; d < DIM; d++) {
            const double ud = (d == dir) ? Ss : q[1 + d];
            Fh[1 + d] = fma(S, fac * ud - r * q[1 + d], Fh[1 + d]);
        }
        Fh[1 + DIM] = fma(S, feS - E, Fh[1 + DIM]);
    }
    return Ss;
}

template <int DIM, int NS, int TX, int TY, int TZ, int MODE>
__global__ void __launch_bounds__(TileGeom<DIM, TX, TY, TZ>::THREADS,
                                  stencil_min_blocks<DIM, NS, TX, TY, TZ>())
stencil_kernel(NetParams P, int limiter, long long Ntot, const BoxDev* __restrict__ boxes,
               const TileDev* __restrict__ tiles, const double* __restrict__ U, double* __restrict__ Aout,
               RhsArgs ra) {
    using G = TileGeom<DIM, TX, TY, TZ>;
    constexpr int NV = 2 + DIM + NS;
    constexpr int NH = 2 + DIM;   // hydrodynamic fields (rho, u, p / rho, rho u, rho E)
    extern __shared__ double smem[];
    double* sq = smem;                 // [NV][NC] primitives
    double* sb = smem + NV * G::NC;    // [NV][NB] half slopes, then face fluxes
    double* sm = sb + NV * G::NB;      // [NB] per face: mass flux / sum of X, times 1/dx

    const TileDev t = tiles[blockIdx.x];
    const BoxDev b = boxes[t.box];
    const int ex = min(TX, b.n[0] - t.o[0]);
    const int ey = DIM >= 2 ? min(TY, b.n[1] - t.o[1]) : 1;
    const int ez = DIM >= 3 ? min(TZ, b.n[2] - t.o[2]) : 1;
    const double g = P.gamma, gm1 = P.gm1, gm1_inv = P.gm1_inv;

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
        const double ir = rcp_nr(rho);
        double ke = 0.0;
        sq[0 * G::NC + s] = rho;
#pragma unroll
        for (int d = 0; d < DIM; d++) {
            const double m = __ldg(U + (1 + d) * Ntot + gi);
            const double u = m * ir;
            sq[(1 + d) * G::NC + s] = u;
            ke = fma(m, u, ke);
        }
        sq[(1 + DIM) * G::NC + s] = gm1 * fma(-0.5, ke, __ldg(U + (1 + DIM) * Ntot + gi));
#pragma unroll
        for (int sp = 0; sp < NS; sp++) sq[(2 + DIM + sp) * G::NC + s] = __ldg(U + (2 + DIM + sp) * Ntot + gi) * ir;
    }
    __syncthreads();

    const int tx = threadIdx.x % TX, ty = (threadIdx.x / TX) % TY, tz = threadIdx.x / (TX * TY);
    const bool own = (threadIdx.x < G::NT) && tx < ex && ty < ey && tz < ez;
    double A[NV];
#pragma unroll
    for (int f = 0; f < NV; f++) A[f] = 0.0;

#pragma unroll
    for (int dir = 0; dir < DIM; dir++) {
        const int e[3] = {ex, ey, ez};
        const int T[3] = {TX, TY, TZ};
        // ---- half slopes of the zones at positions -1..e_dir along dir
        {
            const int S0 = dir == 0 ? TX + 2 : TX, S1 = dir == 1 ? TY + 2 : TY;
            const int nsl = S0 * S1 * (dir == 2 ? TZ + 2 : TZ);
            for (int si = threadIdx.x; si < nsl; si += blockDim.x) {
                int c[3] = {si % S0, (si / S0) % S1, si / (S0 * S1)};
                c[dir] -= 1;
                if (c[dir] > e[dir] || c[(dir + 1) % 3] >= e[(dir + 1) % 3] || c[(dir + 2) % 3] >= e[(dir + 2) % 3])
                    continue;
                int sl[3];
#pragma unroll
                for (int o = 0; o < 3; o++) {
                    int cc[3] = {c[0], c[1], c[2]};
                    cc[dir] += o - 1;
                    sl[o] = slot_of<DIM, TX, TY, TZ>(cc[0], cc[1], cc[2], ey, ez);
                }
#pragma unroll
                for (int f = 0; f < NV; f++)
                    sb[f * G::NB + si] = mc_half_slope(limiter, sq[f * G::NC + sl[0]], sq[f * G::NC + sl[1]],
                                                       sq[f * G::NC + sl[2]]);
            }
        }
        __syncthreads();
        // ---- face fluxes: face i along dir sits between zones i-1 and i
        const int T0 = dir == 0 ? TX + 1 : TX, T1 = dir == 1 ? TY + 1 : TY;
        const int nfaces = T0 * T1 * (dir == 2 ? TZ + 1 : TZ);
        const int S0 = dir == 0 ? TX + 2 : TX, S1 = dir == 1 ? TY + 2 : TY;
        double F[NV];
        double fmi = 0.0;
        int fi_mine = -1;
        {
            const int fi = threadIdx.x;  // THREADS >= faces of every direction
            if (fi < nfaces) {
                const int c0 = fi % T0, c1 = (fi / T0) % T1, c2 = fi / (T0 * T1);
                int c[3] = {c0, c1, c2};
                if (c[0] < (dir == 0 ? ex + 1 : ex) && c[1] < (dir == 1 ? ey + 1 : ey) &&
                    c[2] < (dir == 2 ? ez + 1 : ez)) {
                    fi_mine = fi;
                    int cl[3] = {c0, c1, c2}, cr[3] = {c0, c1, c2};
                    cl[dir] -= 1;
                    const int zl = slot_of<DIM, TX, TY, TZ>(cl[0], cl[1], cl[2], ey, ez);
                    const int zr = slot_of<DIM, TX, TY, TZ>(cr[0], cr[1], cr[2], ey, ez);
                    int sc[3] = {c0, c1, c2};  // slope index of the right zone (position +1 offset)
                    sc[dir] += 1;
                    const int sr = sc[0] + S0 * (sc[1] + S1 * sc[2]);
                    sc[dir] -= 1;
                    const int slf = sc[0] + S0 * (sc[1] + S1 * sc[2]);
                    double qL[NH], qR[NH];
#pragma unroll
                    for (int f = 0; f < NH; f++) {
                        qL[f] = sq[f * G::NC + zl] + sb[f * G::NB + slf];
                        qR[f] = sq[f * G::NC + zr] - sb[f * G::NB + sr];
                    }
                    const double Ss = hllc_hydro<DIM>(g, gm1_inv, dir, qL, qR, F);
                    // species: upwind side of the contact, renormalised
                    const bool lft = nonneg(Ss);
                    const int zu = lft ? zl : zr, su = lft ? slf : sr;
                    // right face of the left zone (+h) or left face of the right zone (-h): the
                    // sign flip on the bit pattern keeps one FP64 add per species
                    const long long flip = lft ? 0ll : SIGN_BIT;
                    double X[NS > 0 ? NS : 1];
                    double sum = 0.0;
#pragma unroll
                    for (int s = 0; s < NS; s++) {
                        const double q = sq[(NH + s) * G::NC + zu], h = sb[(NH + s) * G::NB + su];
                        X[s] = q + bitsd(dbits(h) ^ flip);
                        sum += X[s];
                    }
                    // species flux F_s = fm X_s, fm = F_rho / sum X: the face keeps X_s and
                    // fm / dx, and each zone adds fm_lo X_lo / dx - fm_hi X_hi / dx by two
                    // fused multiply-adds
                    fmi = F[0] * rcp_nr(sum) * b.idx[dir];
#pragma unroll
                    for (int s = 0; s < NS; s++) F[NH + s] = X[s];
                }
            }
        }
        __syncthreads();  // every slope is read: the buffer now takes the fluxes
        if (fi_mine >= 0) {
#pragma unroll
            for (int f = 0; f < NV; f++) sb[f * G::NB + fi_mine] = F[f];
            sm[fi_mine] = fmi;
        }
        __syncthreads();
        if (own) {
            int c[3] = {tx, ty, tz};
            const int lo = c[0] + T0 * (c[1] + T1 * c[2]);
            c[dir] += 1;
            const int hi = c[0] + T0 * (c[1] + T1 * c[2]);
            const double idx = b.idx[dir];
#pragma unroll
            for (int f = 0; f < NH; f++) A[f] = fma(-(sb[f * G::NB + hi] - sb[f * G::NB + lo]), idx, A[f]);
            const double ml = sm[lo], mh = sm[hi];
#pragma unroll
            for (int s = 0; s < NS; s++) {
                A[NH + s] = fma(ml, sb[(NH + s) * G::NB + lo], A[NH + s]);
                A[NH + s] = fma(-mh, sb[(NH + s) * G::NB + hi], A[NH + s]);
            }
        }
        (void)T;
        __syncthreads();
    }

    if (!own) return;
    const long long gi = b.off + (t.o[0] + tx) + (long long)b.n[0] * ((t.o[1] + ty) + (long long)b.n[1] * (t.o[2] + tz));
#pragma unroll
    for (int f = 0; f < NV; f++) Aout[f * Ntot + gi] = A[f];
    if (MODE == STENCIL_A_RHS) {
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
