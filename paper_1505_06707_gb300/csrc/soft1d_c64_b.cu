// complex64 resident 1D step kernels, N = 4096 .. 16384
#include "soft1d_inst.cuh"
namespace soft {
Launch1D soft1d_c64_b(int logn, int loge, int logrm) {
    SOFT1D_CASE(float, 12, 3, 3) SOFT1D_CASE(float, 12, 4, 4)
    SOFT1D_CASE(float, 13, 4, 4) SOFT1D_CASE(float, 13, 5, 4)
    SOFT1D_CASE(float, 14, 5, 4)
    return nullptr;
}
}  // namespace soft
