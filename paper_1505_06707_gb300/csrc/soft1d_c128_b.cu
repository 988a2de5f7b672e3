// complex128 resident 1D step kernels, N = 4096 .. 8192
#include "soft1d_inst.cuh"
namespace soft {
Launch1D soft1d_c128_b(int logn, int loge, int logrm) {
    SOFT1D_CASE(double, 12, 3, 3) SOFT1D_CASE(double, 12, 4, 3)
    SOFT1D_CASE(double, 13, 4, 3) SOFT1D_CASE(double, 13, 3, 3)
    SOFT1D_CASE(double, 14, 5, 3)
    return nullptr;
}
}  // namespace soft
