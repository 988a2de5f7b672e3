// complex64 resident 1D step kernels, N = 64 .. 2048
#include "soft1d_inst.cuh"
namespace soft {
Launch1D soft1d_c64_a(int logn, int loge, int logrm) {
    SOFT1D_CASE(float, 6, 1, 1)
    SOFT1D_CASE(float, 7, 2, 2)
    SOFT1D_CASE(float, 8, 3, 3)
    SOFT1D_CASE(float, 9, 3, 3) SOFT1D_CASE(float, 9, 4, 4)
    SOFT1D_CASE(float, 10, 3, 3) SOFT1D_CASE(float, 10, 4, 4)
    SOFT1D_CASE(float, 11, 3, 3) SOFT1D_CASE(float, 11, 4, 4)
    return nullptr;
}
}  // namespace soft
