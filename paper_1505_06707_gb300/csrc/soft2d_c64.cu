// c64 2D pass kernels (row passes, column pass, y-strip pass), N = 256 .. 2048 per axis
#include "soft2d.cuh"

namespace soft {

int soft2d_row_c64(int logn, int loge, int logrm, int mode, const Geo2D& g, void* psi, int row0,
                    int nrows, const void* tkx, cudaStream_t st) {
#define ROWCASE(LN, LE, LR) \
    if (logn == LN && loge == LE && logrm == LR) return launch_row_t<float, LN, LE, LR>(mode, g, psi, row0, nrows, tkx, st);
    ROWCASE(8, 3, 3) ROWCASE(9, 3, 3) ROWCASE(10, 4, 4) ROWCASE(11, 4, 4)
#undef ROWCASE
    return SOFT_ERR_UNSUPPORTED;
}

int soft2d_col_c64(int logn, int loge, int logrm, const Geo2D& g, void* psi, const void* tky,
                    cudaStream_t st) {
#define COLCASE(LN, LE, LR) \
    if (logn == LN && loge == LE && logrm == LR) return launch_col_t<float, LN, LE, LR, 4>(g, psi, tky, st);
    COLCASE(8, 3, 3) COLCASE(9, 3, 3) COLCASE(10, 5, 4) COLCASE(11, 5, 4)
#undef COLCASE
    return SOFT_ERR_UNSUPPORTED;
}

int soft2d_cny_c64(const Geo2D& g, void* psi, cudaStream_t st) {
    return launch_cny_t<float2, 24>(g, psi, st);
}

}  // namespace soft
