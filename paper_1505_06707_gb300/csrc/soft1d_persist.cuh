// Persistent launch of a mixed-size 1D batch: one CTA of 512 threads per SM
// takes work from a queue ordered longest first until the queue is empty.
// A work item (a pack) is up to G instances of one size, G = 512 / T, each
// advanced by its own warp-aligned group of T threads with a named barrier,
// so every size keeps the thread count and shared memory per instance of its
// one-instance kernel.  The big packs (N = 16384, 2 x 8192) go first; the
// small ones (2 x 4096, 4 x 2048) fill the tail, so the SMs finish together.
#pragma once
#include "soft1d.cuh"

namespace soft {

constexpr int PERSIST_THREADS = 512;

// (LOGN, LOGE, LOGRM) of the kernel's variants, [0] complex64, [1] complex128,
// largest N first (the queue order)
constexpr int PERSIST_CFG[2][4][3] = {{{14, 5, 4}, {13, 5, 4}, {12, 4, 4}, {11, 4, 4}},
                                      {{14, 5, 3}, {13, 4, 3}, {12, 4, 3}, {11, 3, 3}}};

// variant index of a size (-1: not in the persistent kernel), its
// (LOGE, LOGRM) and the instances per CTA
inline int persist_variant(int prec, int logn, int* loge, int* logrm, int* groups) {
    const int p = prec == SOFT_C64 ? 0 : 1;
    for (int v = 0; v < 4; ++v)
        if (PERSIST_CFG[p][v][0] == logn) {
            *loge = PERSIST_CFG[p][v][1];
            *logrm = PERSIST_CFG[p][v][2];
            *groups = PERSIST_THREADS / (1 << (logn - *loge));
            return v;
        }
    return -1;
}

template <typename R, int LOGN, int LOGE, int LOGRM>
struct PVar {
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    static constexpr int LN = LOGN, LE = LOGE, LRM = LOGRM;
    static constexpr int T = K::T;
    static constexpr int G = PERSIST_THREADS / K::T;
    static_assert(G >= 1 && G <= 8 && G * K::T == PERSIST_THREADS, "groups of a CTA");
    static constexpr size_t TWB = sizeof(typename TwT<R>::T) * TwCountT<typename TwT<R>::T, LOGN, LOGRM>::value;
    static constexpr size_t INST = soft1d_inst_smem<R, LOGN, LOGE, LOGRM>();
    static constexpr size_t SMEM = TWB + G * INST;
    static_assert(TWB % 16 == 0 && INST % 16 == 0, "16-byte aligned parts");
};

// one pack: the twiddles of its size into shared memory (the same for every
// instance of that size), then each group advances its instance
template <typename R, class V>
__device__ __forceinline__ void run_pack(const Pack1D& pk, const Inst1D* __restrict__ insts, void* psi,
                                         int64_t nsteps, const double* ftab, int64_t fstride, int* status,
                                         unsigned char* smem) {
    using C = typename CT<R>::C;
    using TWT = typename TwT<R>::T;
    constexpr int TWN = TwCountT<TWT, V::LN, V::LRM>::value;
    TWT* Ws = reinterpret_cast<TWT*>(smem);
    const TWT* __restrict__ W = reinterpret_cast<const TWT*>(insts[pk.first].W);
    copy16(Ws, W, TWN, threadIdx.x, PERSIST_THREADS);
    __syncthreads();
    const int g = threadIdx.x / V::T, tid = threadIdx.x % V::T;
    if (g < pk.count) {
        C* Ss = reinterpret_cast<C*>(smem + V::TWB + g * V::INST);
        C* scan = Ss + (V::K::GM ? 0 : V::K::N);
        const Inst1D& I = insts[pk.first + g];       // read in place (re-loadable, not spilled)
        if constexpr (V::G == 1)
            soft1d_run<R, V::LN, V::LE, V::LRM>(I, psi, nsteps, ftab, fstride, status, Ss, scan, Ws, tid,
                                                BarCTA());
        else
            soft1d_run<R, V::LN, V::LE, V::LRM>(I, psi, nsteps, ftab, fstride, status, Ss, scan, Ws, tid,
                                                BarGroup{1 + g, V::T});
    }
    __syncthreads();    // the next pack reuses the twiddles and the groups' memory
}

template <typename R, class V0, class V1, class V2, class V3>
__global__ void __launch_bounds__(PERSIST_THREADS, 1)
soft1d_persist_kernel(const Pack1D* __restrict__ packs, int npacks, int* __restrict__ counter,
                      const Inst1D* __restrict__ insts, void* __restrict__ psi, int64_t nsteps,
                      const double* __restrict__ ftab, int64_t fstride, int* __restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int next;
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);
        __syncthreads();
        const int p = next;
        __syncthreads();                // read by all before thread 0 takes the next one
        if (p >= npacks) break;
        const Pack1D pk = packs[p];
        switch (pk.var) {
        case 0: run_pack<R, V0>(pk, insts, psi, nsteps, ftab, fstride, status, smem_raw); break;
        case 1: run_pack<R, V1>(pk, insts, psi, nsteps, ftab, fstride, status, smem_raw); break;
        case 2: run_pack<R, V2>(pk, insts, psi, nsteps, ftab, fstride, status, smem_raw); break;
        case 3: run_pack<R, V3>(pk, insts, psi, nsteps, ftab, fstride, status, smem_raw); break;
        default: break;
        }
    }
}

template <class V0, class V1, class V2, class V3>
constexpr size_t persist_smem() {
    size_t m = V0::SMEM;
    if (V1::SMEM > m) m = V1::SMEM;
    if (V2::SMEM > m) m = V2::SMEM;
    if (V3::SMEM > m) m = V3::SMEM;
    return m;
}

// Launch on `ctas` CTAs (0: the kernel's resident capacity on this device);
// with psi == nullptr only the shared-memory attribute is set and ctas_out
// returns that capacity.
template <typename R, class V0, class V1, class V2, class V3>
int launch_persist_t(const Pack1D* packs, int npacks, int* counter, const Inst1D* insts, void* psi,
                     int64_t nsteps, const double* ftab, int64_t fstride, int* status, cudaStream_t st,
                     int* ctas_out) {
    constexpr size_t smem = persist_smem<V0, V1, V2, V3>();
    static_assert(smem + 16 <= 227 * 1024, "shared memory");
    auto k = soft1d_persist_kernel<R, V0, V1, V2, V3>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SOFT_ERR_CUDA;
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, PERSIST_THREADS, smem) != cudaSuccess)
        return SOFT_ERR_CUDA;
    if (per < 1) return SOFT_ERR_UNSUPPORTED;
    const int ctas = nsm * per;
    if (ctas_out) *ctas_out = ctas;
    if (!psi || npacks <= 0) return SOFT_OK;
    k<<<ctas, PERSIST_THREADS, smem, st>>>(packs, npacks, counter, insts, psi, nsteps, ftab, fstride, status);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

}  // namespace soft
