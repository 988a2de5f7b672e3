// The resident 1D split-operator step (Sec. II of Serov & Sergeeva,
// arXiv:1505.06707): one CTA owns one instance; the state lives in shared
// memory for all nsteps steps of a launch.
//
// Per step (after the initial half-kinetic factor of the call):
//   V:  psi *= e^{-iU tau} off the strip block, e^{-iU tau/2} on it
//       (U = U0(z) + E(t+tau/2) xc, Sec. II under Eq. SSFFT)
//   CN: on the block, psi <- 2 M^-1 psi - psi with M = 1 + i tau C/2, which
//       equals (1 + i tau C/2)^-1 (1 - i tau C/2) psi (Sec. II, CN form of
//       e^{-iC tau}); then e^{-iU tau/2} again on the block
//   K:  forward FFT (DIF, digit-reversed output), e^{-i k^2 tau/2}/N in that
//       order, inverse FFT (DIT, natural output).  The half-kinetic factors of
//       consecutive steps are merged; the last step of a launch uses
//       e^{-i k^2 tau/4}.
#pragma once
#include "device_common.cuh"
#include "internal.h"

namespace soft {

// LOGE: log2 of the elements per thread; LOGRM: log2 of the largest pass
// radix (<= 4).  Passes have radix 2^LOGRM except a last, smaller one.
// Diagonal phase tables: complex128 plans store double2; complex64 plans store
// float4 = (hi.re, hi.im, lo.re, lo.im) with hi + lo the FP64 value, applied
// by an FMA chain so that no fixed rounding of the table repeats every step.
template <typename R> struct TabT;
template <> struct TabT<float> { using T = float4; };
template <> struct TabT<double> { using T = double2; };

__device__ __forceinline__ float2 tmul(float2 x, float4 t) {
    const float a = x.x, b = x.y;
    const float re = fmaf(a, t.x, fmaf(-b, t.y, fmaf(a, t.z, -b * t.w)));
    const float im = fmaf(a, t.y, fmaf(b, t.x, fmaf(a, t.w, b * t.z)));
    return make_float2(re, im);
}
__device__ __forceinline__ double2 tmul(double2 x, double2 t) { return cmul(x, t); }

template <typename R, int LOGN, int LOGE, int LOGRM>
struct Cfg1D {
    using C = typename CT<R>::C;
    using TT = typename TabT<R>::T;
    static constexpr int N = 1 << LOGN;
    static constexpr int E = 1 << LOGE;
    static constexpr int T = N / E;
    static constexpr int NFULL = LOGN / LOGRM;
    static constexpr int LOGREM = LOGN % LOGRM;
    static constexpr int NPASS = NFULL + (LOGREM ? 1 : 0);
    static constexpr int CMAX = E / 4 + 2;   // strip rows per thread
    static constexpr int NW = (T + 31) / 32;
    static constexpr int MINB = T >= 512 ? 1 : 512 / T;   // CTAs per SM the registers must allow (128 regs)
    static constexpr size_t SMEM = sizeof(C) * (N + 2 * 32 + E + 4) + 64;
};

// Twiddle tables: for pass P (sub-transform length L, stride s = L/R) and
// every offset off < s, four entries W_L^{off}, W_L^{2 off}, W_L^{4 off},
// W_L^{8 off} (W_L = e^{-2 pi i/L}); a butterfly forms W_L^{m off} for
// m < 16 from the binary digits of m with at most two products.
template <int LOGN, int LOGRM, int P>
struct PassGeom {
    static constexpr int NFULL = LOGN / LOGRM;
    static constexpr int LOGREM = LOGN % LOGRM;
    static constexpr int LOGR = (P < NFULL) ? LOGRM : LOGREM;
    static constexpr int LOGL = LOGN - LOGRM * P;
    static constexpr int S = 1 << (LOGL - LOGR);
    // element offset of this pass's table
    static constexpr int TOFF = PassGeom<LOGN, LOGRM, P - 1>::TOFF + 4 * PassGeom<LOGN, LOGRM, P - 1>::S;
};
template <int LOGN, int LOGRM>
struct PassGeom<LOGN, LOGRM, -1> { static constexpr int TOFF = 0, S = 0; };

template <typename C, int M>
__device__ __forceinline__ C tw_pow(const C* b) {
    static_assert(M >= 1 && M < 16, "radix <= 16");
    if constexpr (M == 1 || M == 2 || M == 4 || M == 8) {
        return b[M == 1 ? 0 : M == 2 ? 1 : M == 4 ? 2 : 3];
    } else {
        constexpr int lo = M & (-M);               // lowest set bit
        return cmul(tw_pow<C, lo>(b), tw_pow<C, M - lo>(b));
    }
}

template <typename C, int RR, int M>
struct StoreFwd {   // y_M = v[bitrev(M)] * W^{M off}, stored at base + M s
    __device__ __forceinline__ static void run(C* S, const C* v, const C* b, int base, int s, bool tw) {
        constexpr int LOGR = (RR == 16) ? 4 : (RR == 8) ? 3 : (RR == 4) ? 2 : (RR == 2) ? 1 : 0;
        C y = v[bitrev_c(M, LOGR)];
        if constexpr (M > 0) { if (tw) y = cmul(y, tw_pow<C, M>(b)); }
        S[swz<C>(base + M * s)] = y;
        if constexpr (M + 1 < RR) StoreFwd<C, RR, M + 1>::run(S, v, b, base, s, tw);
    }
};
template <typename C, int RR, int M>
struct LoadInv {    // v_M = S[base + M s] * conj(W^{M off})
    __device__ __forceinline__ static void run(const C* S, C* v, const C* b, int base, int s, bool tw) {
        C y = S[swz<C>(base + M * s)];
        if constexpr (M > 0) { if (tw) y = cmulc(y, tw_pow<C, M>(b)); }
        v[M] = y;
        if constexpr (M + 1 < RR) LoadInv<C, RR, M + 1>::run(S, v, b, base, s, tw);
    }
};
template <typename C, int RR, int M>
struct StoreNat {   // x_M = v[bitrev(M)] stored at base + M s
    __device__ __forceinline__ static void run(C* S, const C* v, int base, int s) {
        constexpr int LOGR = (RR == 16) ? 4 : (RR == 8) ? 3 : (RR == 4) ? 2 : (RR == 2) ? 1 : 0;
        S[swz<C>(base + M * s)] = v[bitrev_c(M, LOGR)];
        if constexpr (M + 1 < RR) StoreNat<C, RR, M + 1>::run(S, v, base, s);
    }
};

template <typename C, int NB>
__device__ __forceinline__ void load_tw(C* b, const C* __restrict__ t) {
#pragma unroll
    for (int k = 0; k < NB; ++k) b[k] = __ldg(&t[k]);
}

// forward DIF pass P (radix 2^LOGR on sub-transforms of length 2^LOGL)
template <typename R, int LOGN, int LOGE, int LOGRM, int P>
__device__ __forceinline__ void fwd_pass(typename CT<R>::C* S, const typename CT<R>::C* __restrict__ W,
                                         int tid) {
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    using G = PassGeom<LOGN, LOGRM, P>;
    constexpr int RR = 1 << G::LOGR;
    constexpr int L = 1 << G::LOGL;
    constexpr int s = G::S;
    constexpr int NB = G::LOGR;               // twiddle bases needed: 2^0 .. 2^(LOGR-1)
#pragma unroll 1
    for (int u = 0; u < K::E / RR; ++u) {      // one butterfly live at a time
        const int b = tid + u * K::T;
        const int blk = b / s, off = b & (s - 1);
        const int base = blk * L + off;
        C v[RR];
#pragma unroll
        for (int j = 0; j < RR; ++j) v[j] = S[swz<C>(base + j * s)];
        dft_reg<C, RR, -1>(v);
        C tb[4];
        if constexpr (s > 1) load_tw<C, NB>(tb, W + G::TOFF + 4 * off);
        StoreFwd<C, RR, 0>::run(S, v, tb, base, s, s > 1);
    }
}

// inverse DIT pass P (undoes fwd_pass P up to the factor 2^LOGR)
template <typename R, int LOGN, int LOGE, int LOGRM, int P>
__device__ __forceinline__ void inv_pass(typename CT<R>::C* S, const typename CT<R>::C* __restrict__ W,
                                         int tid) {
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    using G = PassGeom<LOGN, LOGRM, P>;
    constexpr int RR = 1 << G::LOGR;
    constexpr int L = 1 << G::LOGL;
    constexpr int s = G::S;
    constexpr int NB = G::LOGR;
#pragma unroll 1
    for (int u = 0; u < K::E / RR; ++u) {      // one butterfly live at a time
        const int b = tid + u * K::T;
        const int blk = b / s, off = b & (s - 1);
        const int base = blk * L + off;
        C v[RR];
        C tb[4];
        if constexpr (s > 1) load_tw<C, NB>(tb, W + G::TOFF + 4 * off);
        LoadInv<C, RR, 0>::run(S, v, tb, base, s, s > 1);
        dft_reg<C, RR, +1>(v);
        StoreNat<C, RR, 0>::run(S, v, base, s);
    }
}

// Whole transforms.  tid is the thread's index within the group of T threads
// that own this transform; every thread of the CTA must call (the passes are
// separated by __syncthreads), so several transforms can share a CTA.
template <typename R, int LOGN, int LOGE, int LOGRM, int P>
__device__ __forceinline__ void fwd_fft(typename CT<R>::C* S, const typename CT<R>::C* W, int tid) {
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    if constexpr (P < K::NPASS) {
        fwd_pass<R, LOGN, LOGE, LOGRM, P>(S, W, tid);
        __syncthreads();
        fwd_fft<R, LOGN, LOGE, LOGRM, P + 1>(S, W, tid);
    }
}
template <typename R, int LOGN, int LOGE, int LOGRM, int P>
__device__ __forceinline__ void inv_fft(typename CT<R>::C* S, const typename CT<R>::C* W, int tid) {
    if constexpr (P >= 0) {
        inv_pass<R, LOGN, LOGE, LOGRM, P>(S, W, tid);
        __syncthreads();
        inv_fft<R, LOGN, LOGE, LOGRM, P - 1>(S, W, tid);
    }
}

// k-space factor (table already in the digit-reversed order of fwd_fft)
template <typename R, int LOGN, int LOGE, int LOGRM>
__device__ __forceinline__ void kmul(typename CT<R>::C* S, const typename TabT<R>::T* __restrict__ tab,
                                     int tid) {
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
#pragma unroll 4
    for (int j = 0; j < K::E; ++j) {
        const int n = tid + j * K::T;
        S[swz<typename K::C>(n)] = tmul(S[swz<typename K::C>(n)], __ldg(&tab[n]));
    }
    __syncthreads();
}

// Crank-Nicolson factor on the strip block (Sec. II, CN form of e^{-iC tau}):
// with M = 1 + i tau C/2 factored on the host (no pivoting) into the
// recurrences y_i = mf_i y_{i-1} + r_i and x_i = mb_i x_{i+1} + g_i y_i, the
// block rows r_i = S[(blk0 + i) mod N] become post(n, 2 x_i - r_i), which is
// (1 + i tau C/2)^{-1} (1 - i tau C/2) r.  Each thread runs a contiguous chunk
// of rows; the chunks are joined by block-wide scans of the affine maps.
// cn holds mf[nb], mb[nb], g[nb].  All T threads must call.
template <typename C, int T, int CMAX, int N, class Post>
__device__ __forceinline__ void strip_cn(C* S, const C* __restrict__ cn, int nb, int blk0, int tid,
                                         C* scan, Post post) {
    const int chunk = (nb + T - 1) / T;          // host guarantees chunk <= CMAX
    const int i0 = tid * chunk;
    C y[CMAX];
    C Mp; Mp.x = 1; Mp.y = 0;
    C yl; yl.x = 0; yl.y = 0;
#pragma unroll
    for (int c = 0; c < CMAX; ++c) {
        const int i = i0 + c;
        if (c < chunk && i < nb) {
            const C rc = S[swz<C>((blk0 + i) & (N - 1))];
            const C m = __ldg(&cn[i]);
            yl = cfma(m, yl, rc);
            Mp = cmul(m, Mp);
            y[c] = yl;
        }
    }
    C carry = affine_carry<C, T, false>(Mp, yl, scan);
    {
        C pr; pr.x = 1; pr.y = 0;
#pragma unroll
        for (int c = 0; c < CMAX; ++c) {
            const int i = i0 + c;
            if (c < chunk && i < nb) {
                pr = cmul(__ldg(&cn[i]), pr);
                y[c] = cfma(pr, carry, y[c]);
            }
        }
    }
    Mp.x = 1; Mp.y = 0;
    C xl; xl.x = 0; xl.y = 0;
#pragma unroll
    for (int c = CMAX - 1; c >= 0; --c) {
        const int i = i0 + c;
        if (c < chunk && i < nb) {
            const C m = __ldg(&cn[nb + i]);
            const C g = __ldg(&cn[2 * nb + i]);
            xl = cfma(m, xl, cmul(g, y[c]));
            Mp = cmul(m, Mp);
            y[c] = xl;
        }
    }
    carry = affine_carry<C, T, true>(Mp, xl, scan);
    C pr; pr.x = 1; pr.y = 0;
#pragma unroll
    for (int c = CMAX - 1; c >= 0; --c) {
        const int i = i0 + c;
        if (c < chunk && i < nb) {
            pr = cmul(__ldg(&cn[nb + i]), pr);
            const C xv = cfma(pr, carry, y[c]);
            const int n = (blk0 + i) & (N - 1);
            const C rc = S[swz<C>(n)];
            S[swz<C>(n)] = post(n, cmk<C>(2 * xv.x - rc.x, 2 * xv.y - rc.y));
        }
    }
}

__device__ __forceinline__ void sincos_r(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ void sincos_r(double a, double* s, double* c) { sincos(a, s, c); }

template <typename R, int LOGN, int LOGE, int LOGRM>
__global__ void __launch_bounds__(Cfg1D<R, LOGN, LOGE, LOGRM>::T, Cfg1D<R, LOGN, LOGE, LOGRM>::MINB)
soft1d_kernel(const Inst1D* __restrict__ insts, void* __restrict__ psi_base, int64_t nsteps,
              const double* __restrict__ ftab_base, int64_t ftab_stride, int* __restrict__ status)
{
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    constexpr int N = K::N, T = K::T, E = K::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* S = reinterpret_cast<C*>(smem_raw);
    C* scan = S + N;                 // 2*32 complex
    C* fr = scan + 64;               // E complex: field ratio powers
    C* fc = fr + E;                  // 4 complex: clamped field phases

    const Inst1D I = insts[blockIdx.x];
    C* __restrict__ g_psi = reinterpret_cast<C*>(psi_base) + I.off;
    const C* __restrict__ W = reinterpret_cast<const C*>(I.W);
    using TT = typename K::TT;
    const TT* __restrict__ TK = reinterpret_cast<const TT*>(I.TK);
    const TT* __restrict__ TKh = reinterpret_cast<const TT*>(I.TKh);
    const TT* __restrict__ TV = reinterpret_cast<const TT*>(I.TV);
    const C* __restrict__ cn = reinterpret_cast<const C*>(I.cn);
    const int tid = threadIdx.x;
    const int nb = I.nb, blk0 = I.blk0;

    // load the state
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int n = tid + j * T;
        S[swz<C>(n)] = g_psi[n];
    }
    __syncthreads();

    // first half-kinetic factor of this call
    fwd_fft<R, LOGN, LOGE, LOGRM, 0>(S, W, tid);
    kmul<R, LOGN, LOGE, LOGRM>(S, TKh, tid);
    inv_fft<R, LOGN, LOGE, LOGRM, K::NPASS - 1>(S, W, tid);

    const double* __restrict__ ftab = I.has_field ? ftab_base + (int64_t)I.fcls * ftab_stride : nullptr;
    for (int64_t step = 0; step < nsteps; ++step) {
        // ---- field phase of this step: f_half(x) = exp(-i alpha xc), alpha = tau E(t+tau/2)/2
        R al = 0;
        if (I.has_field) {
            al = (R)(0.5 * I.tau * I.E0 * __ldg(&ftab[step]));
            if (tid < E) {                    // ratio powers exp(-i al j T h)
                R sv, cv; sincos_r(-al * ((R)(tid * T) * (R)I.h), &sv, &cv);
                fr[tid] = cmk<C>(cv, sv);
            }
            if (tid == 0) {
                R sv, cv;
                sincos_r(-al * (R)I.R0, &sv, &cv);
                fc[0] = cmk<C>(cv, sv);      // x >= R0
                fc[1] = cmk<C>(cv, -sv);     // x <= -R0
            }
            __syncthreads();
        }
        // ---- V on every point: full factor off the block, half on it
        {
            C base; base.x = 1; base.y = 0;
            if (I.has_field) {
                R sv, cv; sincos_r(-al * ((R)I.x0 + (R)tid * (R)I.h), &sv, &cv);
                base = cmk<C>(cv, sv);
            }
#pragma unroll 4
            for (int j = 0; j < E; ++j) {
                const int n = tid + j * T;
                C v = tmul(S[swz<C>(n)], __ldg(&TV[n]));
                const bool inblk = ((n - blk0) & (N - 1)) < nb;
                if (I.has_field) {
                    C f = cmul(base, fr[j]);
                    if (inblk) {
                        if (n >= I.iR) f = fc[0];
                        else if (n < I.iL) f = fc[1];
                    } else {
                        f = cmul(f, f);
                    }
                    v = cmul(v, f);
                }
                S[swz<C>(n)] = v;
            }
        }
        __syncthreads();
        // ---- Crank-Nicolson on the strip block, then the second e^{-iU tau/2}
        if (nb > 0) {
            strip_cn<C, T, K::CMAX, N>(S, cn, nb, blk0, tid, scan, [&](int n, C v) {
                v = tmul(v, __ldg(&TV[n]));
                if (I.has_field) {
                    C f;
                    if (n >= I.iR) f = fc[0];
                    else if (n < I.iL) f = fc[1];
                    else {
                        R sv, cv;
                        sincos_r(-al * ((R)I.x0 + (R)n * (R)I.h), &sv, &cv);
                        f = cmk<C>(cv, sv);
                    }
                    v = cmul(v, f);
                }
                return v;
            });
            __syncthreads();
        }
        // ---- kinetic: forward FFT, e^{-iK tau} (or tau/2 on the last step), inverse FFT
        fwd_fft<R, LOGN, LOGE, LOGRM, 0>(S, W, tid);
        kmul<R, LOGN, LOGE, LOGRM>(S, step + 1 < nsteps ? TK : TKh, tid);
        inv_fft<R, LOGN, LOGE, LOGRM, K::NPASS - 1>(S, W, tid);
    }

    // store
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int n = tid + j * T;
        g_psi[n] = S[swz<C>(n)];
    }
    if (tid == 0 && status) {
        const C v = S[0];
        if (!(isfinite((double)v.x) && isfinite((double)v.y))) atomicOr(status, 1);
    }
}

template <typename R, int LOGN, int LOGE, int LOGRM>
int launch_soft1d_t(const Inst1D* d_inst, int count, void* psi, int64_t nsteps,
                    const double* ftab, int64_t ftab_stride, int* d_status, cudaStream_t st,
                    size_t* smem_out)
{
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    auto kern = soft1d_kernel<R, LOGN, LOGE, LOGRM>;
    const size_t smem = K::SMEM;
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return SOFT_ERR_CUDA;
    }
    if (smem_out) *smem_out = smem;
    if (count <= 0) return SOFT_OK;
    kern<<<count, K::T, smem, st>>>(d_inst, psi, nsteps, ftab, ftab_stride, d_status);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

}  // namespace soft
