// 2D split-operator step and the stationary PCG solve (entry points).
#include "plan_internal.h"

using namespace soft;

namespace soft {
struct Plan2D {};
}  // namespace soft

int create_2d(const soft_grid*, const double*, double, double, double, const soft_options&,
              soft_plan**) {
    return SOFT_ERR_UNSUPPORTED;
}
int soft_plan::step_2d(void*, int64_t, double*, cudaStream_t) { return SOFT_ERR_UNSUPPORTED; }
int64_t soft_plan::points_2d() const { return 0; }
void soft_plan::free_2d() { delete p2; p2 = nullptr; }

extern "C" {
int sse_pcg_solve(soft_plan*, const double*, int, const void*, void*, double, int, int, int*,
                  double*, void*) {
    return SOFT_ERR_UNSUPPORTED;
}
int sse_apply_A(soft_plan*, double, const void*, void*, void*) { return SOFT_ERR_UNSUPPORTED; }
int sse_apply_precond(soft_plan*, double, int, const void*, void*, void*) {
    return SOFT_ERR_UNSUPPORTED;
}
}
