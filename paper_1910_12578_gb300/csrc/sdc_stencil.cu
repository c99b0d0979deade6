// sdc_stencil.cu -- instantiations and launch of the advective-term kernel
// (paper section 2, Eq. 1) with the fused right-hand side of Eq. sdc:general.
#include "sdc_launch.h"
#include "sdc_stencil_split.cuh"

namespace sdcd {

#define SDC_STENCIL_CASES(X) \
    X(1, 2)                  \
    X(1, 5)                  \
    X(3, 2)                  \
    X(3, 3)                  \
    X(3, 4)                  \
    X(3, 5)                  \
    X(3, 7)                  \
    X(3, 13)

// Tile shapes (variant V, chosen by the autotuner): 1D lines of 64 zones; in 3D
// cubes of 8^3 (one face per thread in every direction; V = 0) or 8 x 8 x 4
// (V = 1, and the only shape when 8^3 primitives and slopes would not fit in
// shared memory with many species).
template <int DIM, int NS, int V> struct Tile;
template <int NS, int V> struct Tile<1, NS, V> { static constexpr int X = 64, Y = 1, Z = 1; };
template <int NS, int V> struct Tile<3, NS, V> {
    static constexpr int X = 8, Y = 8, Z = (NS <= 7 && V == 0 ? 8 : 4);
};

template <int DIM, int NS, int V>
constexpr size_t smem_bytes() {
    using G = TileGeom<DIM, Tile<DIM, NS, V>::X, Tile<DIM, NS, V>::Y, Tile<DIM, NS, V>::Z>;
    return sizeof(double) * ((size_t)(2 + DIM + NS) * (G::NC + G::NB) + G::NB);
}

// 3D: the tile shapes, then the direction-split passes (stencil_split_kernel)
// as the last variant
int stencil_variants(int dim, int nspec) { return dim == 3 ? (nspec <= 7 ? 3 : 2) : 1; }

int stencil_split_variant(int dim, int nspec) { return dim == 3 ? stencil_variants(dim, nspec) - 1 : -1; }

bool stencil_supported(int dim, int nspec) {
#define X(d, ns) \
    if (dim == d && nspec == ns) return true;
    SDC_STENCIL_CASES(X)
#undef X
    return false;
}

void stencil_tile(int dim, int nspec, int variant, int t[3]) {
    t[0] = 64; t[1] = 1; t[2] = 1;
#define X(d, ns)                                                                                   \
    if (dim == d && nspec == ns) {                                                                 \
        if (variant == 1 && variant != stencil_split_variant(d, ns)) {                             \
            t[0] = Tile<d, ns, 1>::X; t[1] = Tile<d, ns, 1>::Y; t[2] = Tile<d, ns, 1>::Z;          \
        } else {                                                                                   \
            t[0] = Tile<d, ns, 0>::X; t[1] = Tile<d, ns, 0>::Y; t[2] = Tile<d, ns, 0>::Z;          \
        }                                                                                          \
    }
    SDC_STENCIL_CASES(X)
#undef X
}

size_t stencil_smem_bytes(int dim, int nspec, int variant) {
#define X(d, ns) \
    if (dim == d && nspec == ns) return variant == 1 ? smem_bytes<d, ns, 1>() : smem_bytes<d, ns, 0>();
    SDC_STENCIL_CASES(X)
#undef X
    return 0;
}

template <int d, int ns, int V>
cudaError_t prepare_one() {
    constexpr int TX = Tile<d, ns, V>::X, TY = Tile<d, ns, V>::Y, TZ = Tile<d, ns, V>::Z;
    cudaError_t e = cudaFuncSetAttribute(stencil_kernel<d, ns, TX, TY, TZ, STENCIL_A>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<d, ns, V>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(stencil_kernel<d, ns, TX, TY, TZ, STENCIL_A_RHS>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<d, ns, V>());
}

// the direction-split passes (3D): x pass (reads U, writes the primitives),
// y pass, z pass (finishes A, with or without the rhs)
#define SDC_SPLIT_CASES(X) \
    X(2)                   \
    X(3)                   \
    X(4)                   \
    X(5)                   \
    X(7)                   \
    X(13)

template <int ns, int D, bool FIRST, bool LAST, int MODE>
cudaError_t prepare_split_one() {
    return cudaFuncSetAttribute(stencil_split_kernel<ns, D, FIRST, LAST, MODE>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)split_smem_bytes<ns, D>());
}

template <int ns>
cudaError_t prepare_split() {
    cudaError_t e;
    if ((e = prepare_split_one<ns, 0, true, false, STENCIL_A>()) != cudaSuccess) return e;
    if ((e = prepare_split_one<ns, 1, false, false, STENCIL_A>()) != cudaSuccess) return e;
    if ((e = prepare_split_one<ns, 2, false, true, STENCIL_A>()) != cudaSuccess) return e;
    return prepare_split_one<ns, 2, false, true, STENCIL_A_RHS>();
}

cudaError_t stencil_prepare(int dim, int nspec) {
    cudaError_t e = cudaErrorInvalidValue;
#define X(d, ns)                                                          \
    if (dim == d && nspec == ns) {                                        \
        e = prepare_one<d, ns, 0>();                                      \
        if (e == cudaSuccess && stencil_variants(d, ns) > 1 && stencil_split_variant(d, ns) != 1) \
            e = prepare_one<d, ns, 1>();                                  \
    }
    SDC_STENCIL_CASES(X)
#undef X
    if (e != cudaSuccess || dim != 3) return e;
#define X(ns) \
    if (nspec == ns) return prepare_split<ns>();
    SDC_SPLIT_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

void split_tile_shape(int D, int t[3]) {
    t[0] = t[1] = t[2] = 1;
    const int L = D == 0 ? SplitShape<0>::L : (D == 1 ? SplitShape<1>::L : SplitShape<2>::L);
    const int NL = D == 0 ? SplitShape<0>::NL : (D == 1 ? SplitShape<1>::NL : SplitShape<2>::NL);
    t[D] = L;
    t[D == 0 ? 1 : 0] = NL;
}

template <int ns>
cudaError_t launch_split(const NetParams& P, int limiter, long long Ntot, const BoxDev* boxes,
                         const TileDev* const* tiles, const int* ntiles, const double* U, double* prim, double* A,
                         int mode, const RhsArgs& ra, cudaStream_t st) {
    RhsArgs none = ra;
    if (ntiles[0] > 0)
        stencil_split_kernel<ns, 0, true, false, STENCIL_A>
            <<<ntiles[0], SplitGeom<0>::THREADS, split_smem_bytes<ns, 0>(), st>>>(P, limiter, Ntot, boxes, tiles[0],
                                                                                  U, prim, A, none);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ntiles[1] > 0)
        stencil_split_kernel<ns, 1, false, false, STENCIL_A>
            <<<ntiles[1], SplitGeom<1>::THREADS, split_smem_bytes<ns, 1>(), st>>>(P, limiter, Ntot, boxes, tiles[1],
                                                                                  U, prim, A, none);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ntiles[2] > 0) {
        if (mode == STENCIL_A_RHS)
            stencil_split_kernel<ns, 2, false, true, STENCIL_A_RHS>
                <<<ntiles[2], SplitGeom<2>::THREADS, split_smem_bytes<ns, 2>(), st>>>(P, limiter, Ntot, boxes,
                                                                                      tiles[2], U, prim, A, ra);
        else
            stencil_split_kernel<ns, 2, false, true, STENCIL_A>
                <<<ntiles[2], SplitGeom<2>::THREADS, split_smem_bytes<ns, 2>(), st>>>(P, limiter, Ntot, boxes,
                                                                                      tiles[2], U, prim, A, none);
    }
    return cudaGetLastError();
}

cudaError_t launch_stencil_split(const NetParams& P, int limiter, long long Ntot, const BoxDev* boxes,
                                 const TileDev* const* tiles, const int* ntiles, const double* U, double* prim,
                                 double* A, int mode, const RhsArgs& ra, cudaStream_t st) {
    if (!prim) return cudaErrorInvalidValue;
#define X(ns) \
    if (P.nspec == ns) return launch_split<ns>(P, limiter, Ntot, boxes, tiles, ntiles, U, prim, A, mode, ra, st);
    SDC_SPLIT_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

template <int d, int ns, int V>
cudaError_t launch_one(const NetParams& P, int limiter, long long Ntot, const BoxDev* boxes, const TileDev* tiles,
                       int ntiles, const double* U, double* A, int mode, const RhsArgs& ra, cudaStream_t st) {
    constexpr int TX = Tile<d, ns, V>::X, TY = Tile<d, ns, V>::Y, TZ = Tile<d, ns, V>::Z;
    constexpr int NTH = TileGeom<d, TX, TY, TZ>::THREADS;
    const size_t sm = smem_bytes<d, ns, V>();
    if (mode == STENCIL_A)
        stencil_kernel<d, ns, TX, TY, TZ, STENCIL_A><<<ntiles, NTH, sm, st>>>(P, limiter, Ntot, boxes, tiles, U, A, ra);
    else
        stencil_kernel<d, ns, TX, TY, TZ, STENCIL_A_RHS>
            <<<ntiles, NTH, sm, st>>>(P, limiter, Ntot, boxes, tiles, U, A, ra);
    return cudaGetLastError();
}

cudaError_t launch_stencil(const NetParams& P, int dim, int limiter, long long Ntot, const BoxDev* boxes,
                           const TileDev* tiles, int ntiles, const double* U, double* A, int mode,
                           const RhsArgs& ra, cudaStream_t st, int variant) {
    if (ntiles <= 0) return cudaSuccess;
#define X(d, ns)                                                                                      \
    if (dim == d && P.nspec == ns) {                                                                  \
        if (variant == 1 && stencil_split_variant(d, ns) != 1)                                       \
            return launch_one<d, ns, 1>(P, limiter, Ntot, boxes, tiles, ntiles, U, A, mode, ra, st);  \
        return launch_one<d, ns, 0>(P, limiter, Ntot, boxes, tiles, ntiles, U, A, mode, ra, st);      \
    }
    SDC_STENCIL_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace sdcd
