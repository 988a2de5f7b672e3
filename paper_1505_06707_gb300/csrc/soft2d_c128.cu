// c128 pass kernels of the 2D and 3D steps (row passes, strided line passes,
// strip CN along a strided axis), N = 64 .. 2048 per axis
#include "soft2d.cuh"

namespace soft {

int soft2d_row_c128(int logn, int loge, int logrm, int mode, const Geo2D& g, void* psi, int row0,
                    int nrows, const void* tkx, const int* rows, cudaStream_t st) {
#define ROWCASE(LN, LE, LR)                                                                  \
    if (logn == LN && loge == LE && logrm == LR)                                             \
        return launch_row_t<double, LN, LE, LR>(mode, g, psi, row0, nrows, tkx, rows, st);
    ROWCASE(6, 1, 1) ROWCASE(7, 2, 2) ROWCASE(8, 3, 3) ROWCASE(9, 3, 3) ROWCASE(10, 3, 3) ROWCASE(11, 3, 3)
#undef ROWCASE
    return SOFT_ERR_UNSUPPORTED;
}

int soft2d_col_c128(int logn, int loge, int logrm, const LineGeo& g, int planes, void* psi,
                    const void* tky, cudaStream_t st) {
#define COLCASE(LN, LE, LR) \
    if (logn == LN && loge == LE && logrm == LR) return launch_col_t<double, LN, LE, LR, 2>(g, planes, psi, tky, st);
    COLCASE(6, 1, 1) COLCASE(7, 2, 2) COLCASE(8, 3, 3) COLCASE(9, 3, 3) COLCASE(10, 3, 3) COLCASE(11, 3, 3)
#undef COLCASE
    return SOFT_ERR_UNSUPPORTED;
}

int soft2d_cny_c128(const CnGeo& g, int planes, void* psi, cudaStream_t st) {
    return launch_cny_t<double2, 24>(g, planes, psi, st);
}

}  // namespace soft
