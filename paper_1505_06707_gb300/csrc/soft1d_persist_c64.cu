// Persistent mixed-size batch kernel, complex64: N = 16384, 8192, 4096, 2048
// with 1, 2, 2 and 4 instances per CTA.
#include "soft1d_persist.cuh"

namespace soft {
template <int I>
using V = PVar<float, PERSIST_CFG[0][I][0], PERSIST_CFG[0][I][1], PERSIST_CFG[0][I][2]>;

int launch_persist_c64(const Pack1D* packs, int npacks, int* counter, const Inst1D* insts, void* psi,
                       int64_t nsteps, const double* ftab, int64_t fstride, int* status, cudaStream_t st,
                       int* ctas_out) {
    return launch_persist_t<float, V<0>, V<1>, V<2>, V<3>>(packs, npacks, counter, insts, psi, nsteps, ftab, fstride,
                                                   status, st, ctas_out);
}
}  // namespace soft
