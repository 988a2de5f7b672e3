// complex128 resident 1D step kernels, N = 64 .. 2048
#include "soft1d_inst.cuh"
namespace soft {
Launch1D soft1d_c128_a(int logn, int loge, int logrm) {
    SOFT1D_CASE(double, 6, 1, 1)
    SOFT1D_CASE(double, 7, 2, 2)
    SOFT1D_CASE(double, 8, 3, 3)
    SOFT1D_CASE(double, 9, 3, 3)
    SOFT1D_CASE(double, 10, 3, 3) SOFT1D_CASE(double, 10, 4, 3)
    SOFT1D_CASE(double, 11, 3, 3) SOFT1D_CASE(double, 11, 4, 3)
    return nullptr;
}
}  // namespace soft
