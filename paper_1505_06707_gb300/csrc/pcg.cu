// Stationary ECS equation (Sec. III): entry points (filled in with the PCG kernels).
#include "plan_internal.h"

using namespace soft;

void Plan2D::free_pcg() {}

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
