// Explicit instantiation helper: each translation unit includes this with
// SOFT1D_R (float/double) and a list of (LOGN, LOGE) pairs, and exports one
// dispatcher returning the launcher for a pair.
#pragma once
#include "soft1d.cuh"

namespace soft {
using Launch1D = int (*)(const Inst1D*, int, void*, int64_t, const double*, int64_t, int*,
                         cudaStream_t, size_t*);
}  // namespace soft

#define SOFT1D_CASE(R, LN, LE, LRM) \
    if (logn == LN && loge == LE && logrm == LRM) return &launch_soft1d_t<R, LN, LE, LRM>;
