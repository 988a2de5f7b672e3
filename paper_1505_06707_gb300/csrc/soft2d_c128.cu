// c128 pass kernels of the 2D and 3D steps (row passes, strided line passes,
// strip CN along a strided axis), N = 64 .. 2048 per axis
#include "soft2d.cuh"

namespace soft {

int soft2d_row_c128(int logn, int loge, int logrm, int mode, const Geo2D& g, void* psi, int nrows,
                    const void* tkx, cudaStream_t st) {
#define ROWCASE(LN, LE, LR) \
    if (logn == LN && loge == LE && logrm == LR) return launch_row_t<double, LN, LE, LR>(mode, g, psi, nrows, tkx, st);
    ROWCASE(6, 1, 1) ROWCASE(7, 2, 2) ROWCASE(8, 3, 3) ROWCASE(9, 3, 3) ROWCASE(10, 3, 3) ROWCASE(11, 3, 3)
#undef ROWCASE
    return SOFT_ERR_UNSUPPORTED;
}

int soft2d_col_c128(int logn, int loge, int logrm, int mode, const LineGeo& g, int planes, void* psi,
                    const void* tky, cudaStream_t st) {
#define COLCASE(LN, LE, LR) \
    if (logn == LN && loge == LE && logrm == LR) return launch_col_t<double, LN, LE, LR, 2>(mode, g, planes, psi, tky, st);
    COLCASE(6, 1, 1) COLCASE(7, 2, 2) COLCASE(8, 3, 3) COLCASE(9, 3, 3) COLCASE(10, 3, 3) COLCASE(11, 3, 3)
#undef COLCASE
    return SOFT_ERR_UNSUPPORTED;
}

// strip rows the column pass of a configuration can take (0: not built)
int soft2d_col_strip_capacity_c128(int logn, int loge, int logrm) {
    if (logn == 6 && loge == 1 && logrm == 1) return col_strip_capacity<double, 6, 1, 1>();
    if (logn == 7 && loge == 2 && logrm == 2) return col_strip_capacity<double, 7, 2, 2>();
    if (logn == 8 && loge == 3 && logrm == 3) return col_strip_capacity<double, 8, 3, 3>();
    if (logn == 9 && loge == 3 && logrm == 3) return col_strip_capacity<double, 9, 3, 3>();
    if (logn == 10 && loge == 3 && logrm == 3) return col_strip_capacity<double, 10, 3, 3>();
    if (logn == 11 && loge == 3 && logrm == 3) return col_strip_capacity<double, 11, 3, 3>();
    return 0;
}

int soft2d_cny_c128(const CnGeo& g, int planes, void* psi, cudaStream_t st) {
    return launch_cny_t<double2>(g, planes, psi, st);
}

}  // namespace soft
