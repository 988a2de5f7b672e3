// Persistent mixed-size batch kernel, complex128: N = 16384 (state in its own
// buffer), 8192, 4096, 2048 with 1, 1, 2 and 2 instances per CTA.
#include "soft1d_persist.cuh"

namespace soft {
template <int I>
using V = PVar<double, PERSIST_CFG[1][I][0], PERSIST_CFG[1][I][1], PERSIST_CFG[1][I][2]>;

int launch_persist_c128(const Pack1D* packs, int npacks, int* counter, const Inst1D* insts, void* psi,
                        int64_t nsteps, const double* ftab, int64_t fstride, int* status, cudaStream_t st,
                        int* ctas_out) {
    return launch_persist_t<double, V<0>, V<1>, V<2>, V<3>>(packs, npacks, counter, insts, psi, nsteps, ftab, fstride,
                                                    status, st, ctas_out);
}
}  // namespace soft

namespace soft {
int launch_persist_c64(const Pack1D* packs, int npacks, int* counter, const Inst1D* insts, void* psi,
                       int64_t nsteps, const double* ftab, int64_t fstride, int* status, cudaStream_t st,
                       int* ctas_out);

int launch_persist(int prec, const void* packs, int npacks, int* counter, const Inst1D* insts, void* psi,
                   int64_t nsteps, const double* ftab, int64_t fstride, int* status, cudaStream_t st,
                   int* ctas_out) {
    const Pack1D* pk = static_cast<const Pack1D*>(packs);
    if (prec == SOFT_C64)
        return launch_persist_c64(pk, npacks, counter, insts, psi, nsteps, ftab, fstride, status, st, ctas_out);
    if (prec == SOFT_C128)
        return launch_persist_c128(pk, npacks, counter, insts, psi, nsteps, ftab, fstride, status, st, ctas_out);
    return SOFT_ERR_UNSUPPORTED;
}

int persist_config(int prec, int logn, int* loge, int* logrm, int* groups) {
    return persist_variant(prec, logn, loge, logrm, groups);
}
}  // namespace soft
