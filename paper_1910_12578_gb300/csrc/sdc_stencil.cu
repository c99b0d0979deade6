// sdc_stencil.cu -- instantiations and launch of the advective-term kernel
// (paper section 2, Eq. 1) with the fused right-hand side of Eq. sdc:general.
#include "sdc_launch.h"

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
    return sizeof(double) * (size_t)(2 + DIM + NS) * (G::NC + G::NB);
}

int stencil_variants(int dim, int nspec) { return (dim == 3 && nspec <= 7) ? 2 : 1; }

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
        if (variant == 0) { t[0] = Tile<d, ns, 0>::X; t[1] = Tile<d, ns, 0>::Y; t[2] = Tile<d, ns, 0>::Z; } \
        else { t[0] = Tile<d, ns, 1>::X; t[1] = Tile<d, ns, 1>::Y; t[2] = Tile<d, ns, 1>::Z; }     \
    }
    SDC_STENCIL_CASES(X)
#undef X
}

size_t stencil_smem_bytes(int dim, int nspec, int variant) {
#define X(d, ns) \
    if (dim == d && nspec == ns) return variant == 0 ? smem_bytes<d, ns, 0>() : smem_bytes<d, ns, 1>();
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

cudaError_t stencil_prepare(int dim, int nspec) {
#define X(d, ns)                                                     \
    if (dim == d && nspec == ns) {                                   \
        cudaError_t e = prepare_one<d, ns, 0>();                     \
        if (e != cudaSuccess || stencil_variants(d, ns) < 2) return e; \
        return prepare_one<d, ns, 1>();                              \
    }
    SDC_STENCIL_CASES(X)
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
        if (variant == 0 || stencil_variants(d, ns) < 2)                                              \
            return launch_one<d, ns, 0>(P, limiter, Ntot, boxes, tiles, ntiles, U, A, mode, ra, st);  \
        return launch_one<d, ns, 1>(P, limiter, Ntot, boxes, tiles, ntiles, U, A, mode, ra, st);      \
    }
    SDC_STENCIL_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace sdcd
