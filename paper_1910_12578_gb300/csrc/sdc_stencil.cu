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

// Tiles: 1D lines of 64 zones; in 3D cubes of 8^3 (one face per thread in every
// direction), or 8 x 8 x 4 when 8^3 primitives and slopes would not fit in
// shared memory (many species).
template <int DIM, int NS> struct Tile;
template <int NS> struct Tile<1, NS> { static constexpr int X = 64, Y = 1, Z = 1; };
template <int NS> struct Tile<3, NS> {
    static constexpr int X = 8, Y = 8, Z = (NS <= 7 ? 8 : 4);
};

template <int DIM, int NS>
constexpr size_t smem_bytes() {
    using G = TileGeom<DIM, Tile<DIM, NS>::X, Tile<DIM, NS>::Y, Tile<DIM, NS>::Z>;
    return sizeof(double) * (size_t)(2 + DIM + NS) * (G::NC + G::NB);
}

bool stencil_supported(int dim, int nspec) {
#define X(d, ns) \
    if (dim == d && nspec == ns) return true;
    SDC_STENCIL_CASES(X)
#undef X
    return false;
}

void stencil_tile(int dim, int nspec, int t[3]) {
    t[0] = 64; t[1] = 1; t[2] = 1;
#define X(d, ns)                                                                       \
    if (dim == d && nspec == ns) {                                                     \
        t[0] = Tile<d, ns>::X; t[1] = Tile<d, ns>::Y; t[2] = Tile<d, ns>::Z;           \
    }
    SDC_STENCIL_CASES(X)
#undef X
}

size_t stencil_smem_bytes(int dim, int nspec) {
#define X(d, ns) \
    if (dim == d && nspec == ns) return smem_bytes<d, ns>();
    SDC_STENCIL_CASES(X)
#undef X
    return 0;
}

cudaError_t stencil_prepare(int dim, int nspec) {
#define X(d, ns)                                                                                          \
    if (dim == d && nspec == ns) {                                                                        \
        constexpr int TX = Tile<d, ns>::X, TY = Tile<d, ns>::Y, TZ = Tile<d, ns>::Z;                      \
        cudaError_t e = cudaFuncSetAttribute(stencil_kernel<d, ns, TX, TY, TZ, STENCIL_A>,                \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,                 \
                                             (int)smem_bytes<d, ns>());                                   \
        if (e != cudaSuccess) return e;                                                                   \
        return cudaFuncSetAttribute(stencil_kernel<d, ns, TX, TY, TZ, STENCIL_A_RHS>,                     \
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<d, ns>()); \
    }
    SDC_STENCIL_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_stencil(const NetParams& P, int dim, int limiter, long long Ntot, const BoxDev* boxes,
                           const TileDev* tiles, int ntiles, const double* U, double* A, int mode,
                           const RhsArgs& ra, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
#define X(d, ns)                                                                                           \
    if (dim == d && P.nspec == ns) {                                                                       \
        constexpr int TX = Tile<d, ns>::X, TY = Tile<d, ns>::Y, TZ = Tile<d, ns>::Z;                       \
        constexpr int NTH = TileGeom<d, TX, TY, TZ>::THREADS;                                              \
        const size_t sm = smem_bytes<d, ns>();                                                             \
        if (mode == STENCIL_A)                                                                             \
            stencil_kernel<d, ns, TX, TY, TZ, STENCIL_A>                                                   \
                <<<ntiles, NTH, sm, st>>>(P, limiter, Ntot, boxes, tiles, U, A, ra);                       \
        else                                                                                               \
            stencil_kernel<d, ns, TX, TY, TZ, STENCIL_A_RHS>                                               \
                <<<ntiles, NTH, sm, st>>>(P, limiter, Ntot, boxes, tiles, U, A, ra);                       \
        return cudaGetLastError();                                                                         \
    }
    SDC_STENCIL_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace sdcd
