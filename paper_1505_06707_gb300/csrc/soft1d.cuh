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

// Potential phase tables: e^{-iU0 tau} (or its half) stays within |U0 tau| of
// 1, so complex64 plans store d = e^{-iU0 tau} - 1 (FP64 difference rounded to
// FP32, error below |d| 2^-24) and apply psi + psi d; complex128 plans store
// the factor itself.
template <typename R> struct VabT;
template <> struct VabT<float> { using T = float2; };
template <> struct VabT<double> { using T = double2; };
__device__ __forceinline__ float2 vmul(float2 x, float2 d) {
    return make_float2(fmaf(x.x, d.x, fmaf(-x.y, d.y, x.x)), fmaf(x.x, d.y, fmaf(x.y, d.x, x.y)));
}
__device__ __forceinline__ double2 vmul(double2 x, double2 t) { return cmul(x, t); }

// x * conj(hi + lo) for a compensated FP32 value t = (hi.re, hi.im, lo.re, lo.im)
__device__ __forceinline__ float2 tmulc(float2 x, float4 t) {
    const float a = x.x, b = x.y;
    const float re = fmaf(a, t.x, fmaf(b, t.y, fmaf(a, t.z, b * t.w)));
    const float im = fmaf(b, t.x, fmaf(-a, t.y, fmaf(b, t.z, -a * t.w)));
    return make_float2(re, im);
}

// Pass twiddle tables.  Complex128 plans store the four bases W^{2^k off}
// of each offset as double2.  Complex64 plans of the 1D step store each base
// as a compensated float4 (hi + lo = the FP64 value) and apply W^{M off} as
// one compensated multiply per set bit of M: forming the product of rounded
// bases (or rounding any stored twiddle) leaves |w| != 1 by up to ~1e-7,
// and since the forward and the inverse FFT apply the same twiddle to the
// same position, that modulus error returns unchanged in every step and the
// state drifts linearly in time.  With compensated factors the modulus is
// exact to ~2^-48 and only the data's own roundings remain.
// Complex128 plans of the 1D step store, for passes with a stride of at
// most TWFULL_MAXS, every twiddle W^{M off} (M = 1 .. R-1) instead of the
// four bases: the products of bases cost 16 of the ~100 FP64 instructions
// of a radix-8 butterfly, and the kernel is bound by the FP64 pipe.  Passes
// with a larger stride keep the bases (their full table would not fit in
// shared memory).  The complex64 line passes of the 2D and 3D steps use the
// same layout with float2 entries.
template <typename C> struct TwFull { C v; };
using TwFullD = TwFull<double2>;
using TwFullF = TwFull<float2>;

template <typename R> struct TwT;
template <> struct TwT<float> { using T = float4; };
template <> struct TwT<double> { using T = TwFullD; };

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
    // state larger than a CTA's shared memory (complex128, N = 16384): the
    // step kernel works on the instance's own buffer in global memory (L2
    // resident while the CTA runs; such plans are bound by FP64 arithmetic)
    static constexpr bool GM = sizeof(C) * N > 160 * 1024;
};

// Twiddle tables: for pass P (sub-transform length L, stride s = L/R) four
// rows of s entries, row k holding W_L^{2^k off} for off < s (W_L =
// e^{-2 pi i/L}), so the lanes of a warp read consecutive entries of a row; a
// butterfly forms W_L^{m off} for m < 16 from the binary digits of m with at
// most two products.
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

// y * W^{M off} (fwd) and y * conj(W^{M off}) (inv) from the bases b[k] =
// W^{2^k off}: plain bases (TW = C) through one product twiddle, compensated
// FP32 bases (TW = float4) by one compensated multiply per set bit of M
template <typename C, typename TW, int M, bool FULL = false> struct TwMul {
    __device__ __forceinline__ static C fwd(C y, const C* b) { return cmul(y, tw_pow<C, M>(b)); }
    __device__ __forceinline__ static C inv(C y, const C* b) { return cmulc(y, tw_pow<C, M>(b)); }
};
// full tables: full passes hold b[M - 1] = W^{M off}; the other passes hold
// W^{M off} for M = 1 .. 4, and W^{M off} = W^{4 off} W^{(M-4) off} above
// (radix 8: one product instead of up to two)
template <typename C, int M> __device__ __forceinline__ C tw_full(const TwFull<C>* b) {
    static_assert(M >= 1 && M < 16, "radix <= 16");
    if constexpr (M <= 4) return b[M - 1].v;
    else return cmul(b[3].v, tw_full<C, M - 4>(b));
}
template <typename C, int M, bool FULL> struct TwMul<C, TwFull<C>, M, FULL> {
    __device__ __forceinline__ static C fwd(C y, const TwFull<C>* b) {
        if constexpr (FULL) return cmul(y, b[M - 1].v);
        else return cmul(y, tw_full<C, M>(b));
    }
    __device__ __forceinline__ static C inv(C y, const TwFull<C>* b) {
        if constexpr (FULL) return cmulc(y, b[M - 1].v);
        else return cmulc(y, tw_full<C, M>(b));
    }
};
template <int M, bool FULL> struct TwMul<float2, float4, M, FULL> {
    __device__ __forceinline__ static float2 fwd(float2 y, const float4* b) {
        if constexpr ((M & 1) != 0) y = tmul(y, b[0]);
        if constexpr ((M & 2) != 0) y = tmul(y, b[1]);
        if constexpr ((M & 4) != 0) y = tmul(y, b[2]);
        if constexpr ((M & 8) != 0) y = tmul(y, b[3]);
        return y;
    }
    __device__ __forceinline__ static float2 inv(float2 y, const float4* b) {
        if constexpr ((M & 1) != 0) y = tmulc(y, b[0]);
        if constexpr ((M & 2) != 0) y = tmulc(y, b[1]);
        if constexpr ((M & 4) != 0) y = tmulc(y, b[2]);
        if constexpr ((M & 8) != 0) y = tmulc(y, b[3]);
        return y;
    }
};

// The element M of a butterfly lives at base + M s; the callers pass
// sb = swz(base) and the offset of element M is the constant swz(M s).
template <typename C, typename TW, int RR, int SS, int M, bool FULL = false>
struct StoreFwd {   // y_M = v[bitrev(M)] * W^{M off}, stored at base + M s
    __device__ __forceinline__ static void run(C* S, const C* v, const TW* b, int sb, bool tw) {
        constexpr int LOGR = (RR == 16) ? 4 : (RR == 8) ? 3 : (RR == 4) ? 2 : (RR == 2) ? 1 : 0;
        C y = v[bitrev_c(M, LOGR)];
        if constexpr (M > 0) { if (tw) y = TwMul<C, TW, M, FULL>::fwd(y, b); }
        S[sb ^ swz<C>(M * SS)] = y;
        if constexpr (M + 1 < RR) StoreFwd<C, TW, RR, SS, M + 1, FULL>::run(S, v, b, sb, tw);
    }
};
template <typename C, typename TW, int RR, int SS, int M, bool FULL = false>
struct LoadInv {    // v_M = S[base + M s] * conj(W^{M off})
    __device__ __forceinline__ static void run(const C* S, C* v, const TW* b, int sb, bool tw) {
        C y = S[sb ^ swz<C>(M * SS)];
        if constexpr (M > 0) { if (tw) y = TwMul<C, TW, M, FULL>::inv(y, b); }
        v[M] = y;
        if constexpr (M + 1 < RR) LoadInv<C, TW, RR, SS, M + 1, FULL>::run(S, v, b, sb, tw);
    }
};
template <typename C, int RR, int SS, int M>
struct StoreNat {   // x_M = v[bitrev(M)] stored at base + M s
    __device__ __forceinline__ static void run(C* S, const C* v, int sb) {
        constexpr int LOGR = (RR == 16) ? 4 : (RR == 8) ? 3 : (RR == 4) ? 2 : (RR == 2) ? 1 : 0;
        S[sb ^ swz<C>(M * SS)] = v[bitrev_c(M, LOGR)];
        if constexpr (M + 1 < RR) StoreNat<C, RR, SS, M + 1>::run(S, v, sb);
    }
};

// SH: the table has been copied to shared memory (plain loads), else it is
// read from global memory through the read-only path
template <typename C, int NB, int ST, bool SH>
__device__ __forceinline__ void load_tw(C* b, const C* __restrict__ t) {
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        if constexpr (SH) b[k] = t[k * ST];
        else b[k] = __ldg(&t[k * ST]);
    }
}

// Twiddle table layout of a pass: offsets and whether the pass stores every
// W^{M off} (FULL) or the four bases, for twiddle type TW.
template <int LOGN, int LOGRM, int P>
struct TwGeomFull {
    using G = PassGeom<LOGN, LOGRM, P>;
    static constexpr bool FULL = G::S > 1 && G::S <= TWFULL_MAXS;
    static constexpr int ROWS = FULL ? (1 << G::LOGR) - 1 : 4;
    static constexpr int TOFF = TwGeomFull<LOGN, LOGRM, P - 1>::TOFF +
                                TwGeomFull<LOGN, LOGRM, P - 1>::ROWS * PassGeom<LOGN, LOGRM, P - 1>::S;
};
template <int LOGN, int LOGRM>
struct TwGeomFull<LOGN, LOGRM, -1> { static constexpr bool FULL = false; static constexpr int ROWS = 0, TOFF = 0; };

template <typename TW> struct TwLay {      // the four bases W^{2^k off} on every pass
    template <int LOGN, int LOGRM, int P> static constexpr bool full() { return false; }
    template <int LOGN, int LOGRM, int P> static constexpr int toff() { return PassGeom<LOGN, LOGRM, P>::TOFF; }
    template <int LOGN, int LOGRM, int P> static constexpr int rows() { return PassGeom<LOGN, LOGRM, P>::LOGR; }
};
template <typename C> struct TwLay<TwFull<C>> {   // every W^{M off}, or M = 1 .. 4 (tw_full)
    template <int LOGN, int LOGRM, int P> static constexpr bool full() { return TwGeomFull<LOGN, LOGRM, P>::FULL; }
    template <int LOGN, int LOGRM, int P> static constexpr int toff() { return TwGeomFull<LOGN, LOGRM, P>::TOFF; }
    template <int LOGN, int LOGRM, int P> static constexpr int rows() {
        constexpr int R = 1 << PassGeom<LOGN, LOGRM, P>::LOGR;
        return TwGeomFull<LOGN, LOGRM, P>::FULL ? R - 1 : (R - 1 < 4 ? R - 1 : 4);
    }
};

// number of twiddle entries of all passes
template <int LOGN, int LOGRM>
struct TwCount {
    static constexpr int NP = LOGN / LOGRM + ((LOGN % LOGRM) ? 1 : 0);
    static constexpr int value = PassGeom<LOGN, LOGRM, NP - 1>::TOFF + 4 * PassGeom<LOGN, LOGRM, NP - 1>::S;
};
// the same for the table layout of twiddle type TW
template <typename TW, int LOGN, int LOGRM>
struct TwCountT { static constexpr int value = TwCount<LOGN, LOGRM>::value; };
template <typename C, int LOGN, int LOGRM>
struct TwCountT<TwFull<C>, LOGN, LOGRM> {
    static constexpr int NP = LOGN / LOGRM + ((LOGN % LOGRM) ? 1 : 0);
    static constexpr int value = TwGeomFull<LOGN, LOGRM, NP - 1>::TOFF +
                                 TwGeomFull<LOGN, LOGRM, NP - 1>::ROWS * PassGeom<LOGN, LOGRM, NP - 1>::S;
};

// forward DIF pass P (radix 2^LOGR on sub-transforms of length 2^LOGL)
template <typename R, int LOGN, int LOGE, int LOGRM, int P, bool SH = false, typename TW = typename CT<R>::C>
__device__ __forceinline__ void fwd_pass(typename CT<R>::C* S, const TW* __restrict__ W, int tid) {
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
        const int sb = swz<C>(blk * L + off);
        C v[RR];
#pragma unroll
        for (int j = 0; j < RR; ++j) v[j] = S[sb ^ swz<C>(j * s)];
        dft_reg<C, RR, -1>(v);
        constexpr bool FULL = TwLay<TW>::template full<LOGN, LOGRM, P>();
        TW tb[FULL ? RR - 1 : 4];
        if constexpr (s > 1)
            load_tw<TW, TwLay<TW>::template rows<LOGN, LOGRM, P>(), s, SH>(
                tb, W + TwLay<TW>::template toff<LOGN, LOGRM, P>() + off);
        StoreFwd<C, TW, RR, s, 0, FULL>::run(S, v, tb, sb, s > 1);
    }
}

// inverse DIT pass P (undoes fwd_pass P up to the factor 2^LOGR)
template <typename R, int LOGN, int LOGE, int LOGRM, int P, bool SH = false, typename TW = typename CT<R>::C>
__device__ __forceinline__ void inv_pass(typename CT<R>::C* S, const TW* __restrict__ W, int tid) {
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
        const int sb = swz<C>(blk * L + off);
        C v[RR];
        constexpr bool FULL = TwLay<TW>::template full<LOGN, LOGRM, P>();
        TW tb[FULL ? RR - 1 : 4];
        if constexpr (s > 1)
            load_tw<TW, TwLay<TW>::template rows<LOGN, LOGRM, P>(), s, SH>(
                tb, W + TwLay<TW>::template toff<LOGN, LOGRM, P>() + off);
        LoadInv<C, TW, RR, s, 0, FULL>::run(S, v, tb, sb, s > 1);
        dft_reg<C, RR, +1>(v);
        StoreNat<C, RR, s, 0>::run(S, v, sb);
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
template <typename R, int LOGN, int LOGE, int LOGRM, int P, int PSTOP = 0>
__device__ __forceinline__ void inv_fft(typename CT<R>::C* S, const typename CT<R>::C* W, int tid) {
    if constexpr (P >= PSTOP) {
        inv_pass<R, LOGN, LOGE, LOGRM, P>(S, W, tid);
        __syncthreads();
        inv_fft<R, LOGN, LOGE, LOGRM, P - 1, PSTOP>(S, W, tid);
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
    C carry = affine_carry<C, T, false>(Mp, yl, scan, tid);
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
    carry = affine_carry<C, T, true>(Mp, xl, scan, tid);
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

// The same solve for the 1D step kernel.  M is complex symmetric (C is,
// Sec. II), so mb_i = mf_{i+1} and one multiplier array serves both sweeps.
// The host lays the coefficients out for coalesced reads: thread t owns rows
// i0 = t*ch .. i0 + ch - 1 (ch = ceil(nb/T)); cn[c*T + t] = mf_{i0+c} for
// c <= ch (0 past the block), cn[(ch+1)*T + c*T + t] = g_{i0+c}, and
// tvs[c*T + t] = TV at row i0 + c.  Every coefficient is read once, before
// the sweep that uses it; the in-chunk products of the carry corrections are
// formed from registers.  post(n, tv, v) gets the row's grid index and potential.
template <typename C, typename VT, int T, int CMAX, int N, class Post, class B = BarCTA>
__device__ __forceinline__ void strip_cn_1d(C* S, const C* __restrict__ cn, const VT* __restrict__ tvs,
                                            int nb, int blk0, int tid, C* scan, Post post, B bar = B()) {
    const int ch = (nb + T - 1) / T;             // host guarantees ch <= CMAX
    const int P1 = (ch + 1) * T;
    const int i0 = tid * ch;
    const int nv = min(ch, nb - i0);             // rows of this thread (may be <= 0)
    C y[CMAX], m[CMAX + 1];
#pragma unroll
    for (int c = 0; c <= CMAX; ++c)
        if (c <= ch) m[c] = __ldg(&cn[c * T + tid]);
    C Mp; Mp.x = 1; Mp.y = 0;
    C yl; yl.x = 0; yl.y = 0;
#pragma unroll
    for (int c = 0; c < CMAX; ++c) {
        if (c < nv) {
            const C rc = S[swz<C>((blk0 + i0 + c) & (N - 1))];
            yl = cfma(m[c], yl, rc);
            Mp = cmul(m[c], Mp);
            y[c] = yl;
        }
    }
    C carry = affine_carry<C, T, false>(Mp, yl, scan, tid, bar);
    {
        C pr; pr.x = 1; pr.y = 0;
#pragma unroll
        for (int c = 0; c < CMAX; ++c) {
            if (c < nv) {
                pr = cmul(m[c], pr);
                y[c] = cfma(pr, carry, y[c]);
            }
        }
    }
    Mp.x = 1; Mp.y = 0;
    C xl; xl.x = 0; xl.y = 0;
#pragma unroll
    for (int c = CMAX - 1; c >= 0; --c) {
        if (c < nv) {
            xl = cfma(m[c + 1], xl, cmul(__ldg(&cn[P1 + c * T + tid]), y[c]));
            Mp = cmul(m[c + 1], Mp);
            y[c] = xl;
        }
    }
    carry = affine_carry<C, T, true>(Mp, xl, scan, tid, bar);
    C pr; pr.x = 1; pr.y = 0;
#pragma unroll
    for (int c = CMAX - 1; c >= 0; --c) {
        if (c < nv) {
            pr = cmul(m[c + 1], pr);
            const C xv = cfma(pr, carry, y[c]);
            const int n = (blk0 + i0 + c) & (N - 1);
            const C rc = S[swz<C>(n)];
            S[swz<C>(n)] = post(n, __ldg(&tvs[c * T + tid]), cmk<C>(2 * xv.x - rc.x, 2 * xv.y - rc.y));
        }
    }
}

__device__ __forceinline__ void sincos_r(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ void sincos_r(double a, double* s, double* c) { sincos(a, s, c); }

// ---------------------------------------------------------------------------
// Pieces of the resident step kernel.  Twiddles are read from a shared-memory
// copy; the last forward pass, the k-space factor and the first inverse pass
// run as one in-register butterfly; the potential factor is applied as the
// last inverse pass stores its outputs.

template <typename R, int LOGN, int LOGRM>
struct Step1D {
    static constexpr int NPASS = LOGN / LOGRM + ((LOGN % LOGRM) ? 1 : 0);
    static constexpr int TWN = TwCountT<typename TwT<R>::T, LOGN, LOGRM>::value;
    static constexpr int LOGR0 = PassGeom<LOGN, LOGRM, 0>::LOGR;   // radix of pass 0
    static constexpr int R0 = 1 << LOGR0;
};

// shared-memory bytes of soft1d_kernel: state, twiddles, scan scratch, field
// phases (E per-butterfly, 16 per-output, 4 clamped, 16 strip rows inside R0,
// 16 per-output squares)
template <typename R, int LOGN, int LOGE, int LOGRM>
__host__ __device__ constexpr size_t soft1d_smem() {
    return sizeof(typename CT<R>::C) *
               ((Cfg1D<R, LOGN, LOGE, LOGRM>::GM ? 0 : (size_t(1) << LOGN)) + 64 + (size_t(1) << LOGE) + 52) +
           sizeof(typename TwT<R>::T) * TwCountT<typename TwT<R>::T, LOGN, LOGRM>::value + 64;
}

template <typename R, int LOGN, int LOGE, int LOGRM, int P, int PEND, typename TW, class B = BarCTA>
__device__ __forceinline__ void fwd_passes(typename CT<R>::C* S, const TW* Ws, int tid, B bar = B()) {
    if constexpr (P < PEND) {
        fwd_pass<R, LOGN, LOGE, LOGRM, P, true>(S, Ws, tid);
        bar.sync();
        fwd_passes<R, LOGN, LOGE, LOGRM, P + 1, PEND>(S, Ws, tid, bar);
    }
}
template <typename R, int LOGN, int LOGE, int LOGRM, int P, int PSTOP, typename TW, class B = BarCTA>
__device__ __forceinline__ void inv_passes(typename CT<R>::C* S, const TW* Ws, int tid, B bar = B()) {
    if constexpr (P >= PSTOP) {
        inv_pass<R, LOGN, LOGE, LOGRM, P, true>(S, Ws, tid);
        bar.sync();
        inv_passes<R, LOGN, LOGE, LOGRM, P - 1, PSTOP>(S, Ws, tid, bar);
    }
}

// last forward pass (stride 1, no twiddles), the k-space table, the first
// inverse pass: butterfly b owns the R consecutive points b*R + m of the
// digit-reversed spectrum, whose factors the table holds at m*(N/R) + b
//
// With SURF, the spectrum entering the k-space factor is also contracted with
// four weight rows sw[r * N + q] (same transposed index q as the table) into
// acc[r] (surface sampling, soft1d_surf_kernel).
//
// TSH: the table has been copied to shared memory (plain loads).
template <typename R, int LOGN, int LOGE, int LOGRM, bool SURF = false, bool TSH = false>
__device__ __forceinline__ void kcenter(typename CT<R>::C* S, const typename TabT<R>::T* __restrict__ tab,
                                        int tid, const typename CT<R>::C* __restrict__ sw = nullptr,
                                        typename CT<R>::C* acc = nullptr) {
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    using G = PassGeom<LOGN, LOGRM, K::NPASS - 1>;
    static_assert(G::S == 1, "the last pass has stride 1");
    constexpr int LOGR = G::LOGR, RR = 1 << LOGR;
    using TT = typename TabT<R>::T;
    constexpr int NU = K::E / RR;
    // the table entries of butterfly u + 1 are requested before butterfly u
    // is computed (radix <= 4: the loads of one butterfly alone would leave
    // the L2 latency exposed)
    constexpr bool PF = RR <= 4 && NU > 1;
    auto ld = [&](int i) -> TT {
        if constexpr (TSH) return tab[i];
        else return __ldg(&tab[i]);
    };
    TT tn[PF ? RR : 1];
    if constexpr (PF) {
#pragma unroll
        for (int m = 0; m < RR; ++m) tn[m] = ld(m * (K::N / RR) + tid);
    }
#pragma unroll 1
    for (int u = 0; u < NU; ++u) {
        const int base = (tid + u * K::T) * RR;
        TT tc[RR];
        if constexpr (PF) {
#pragma unroll
            for (int m = 0; m < RR; ++m) tc[m] = tn[m];
            if (u + 1 < NU) {
#pragma unroll
                for (int m = 0; m < RR; ++m) tn[m] = ld(m * (K::N / RR) + tid + (u + 1) * K::T);
            }
        } else {
#pragma unroll
            for (int m = 0; m < RR; ++m) tc[m] = ld(m * (K::N / RR) + tid + u * K::T);
        }
        const int sb = swz<C>(base);
        C v[RR];
#pragma unroll
        for (int j = 0; j < RR; ++j) v[j] = S[sb ^ swz<C>(j)];
        dft_reg<C, RR, -1>(v);
        if constexpr (SURF) {
#pragma unroll
            for (int m = 0; m < RR; ++m) {
                const int q = m * (K::N / RR) + tid + u * K::T;
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[r] = cfma(v[bitrev_c(m, LOGR)], __ldg(&sw[r * K::N + q]), acc[r]);
            }
        }
        C w[RR];
#pragma unroll
        for (int m = 0; m < RR; ++m) w[m] = tmul(v[bitrev_c(m, LOGR)], tc[m]);
        dft_reg<C, RR, +1>(w);
#pragma unroll
        for (int m = 0; m < RR; ++m) S[sb ^ swz<C>(m)] = w[bitrev_c(m, LOGR)];
    }
}

// Field phases of one step, alpha = tau E(t + tau/2)/2 (the half factor
// exp(-i alpha x)), at fr[]: [u] = exp(-i alpha u T h) for the butterflies of
// the last inverse pass (u < E/R0); [E + m] = exp(-i alpha m (N/R0) h) for
// their outputs (m < R0) and [E + 36 + m] its square; [E + 16], [E + 17] = the clamped values beyond +R0
// and -R0; [E + 20 + k] = exp(-i alpha x_n) at n = iL + k and [E + 28 + k] at
// n = iR - 8 + k (k < 8), the strip rows just inside R0.
template <typename R, int LOGN, int LOGE, int LOGRM>
__device__ __forceinline__ void field_setup(typename CT<R>::C* fr, R al, const Inst1D& I, int tid) {
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    using Q = Step1D<R, LOGN, LOGRM>;
    constexpr int NB = K::E / Q::R0;
    for (int i = tid; i < NB + Q::R0 + 17; i += K::T) {
        R sv, cv;
        if (i < NB) {
            sincos_r(-al * ((R)(i * K::T) * (R)I.h), &sv, &cv);
            fr[i] = cmk<C>(cv, sv);
        } else if (i < NB + Q::R0) {
            const int m = i - NB;
            const R ph = -al * ((R)(m * (K::N / Q::R0)) * (R)I.h);
            sincos_r(ph, &sv, &cv);
            fr[K::E + m] = cmk<C>(cv, sv);
            sincos_r(2 * ph, &sv, &cv);                  // the full step's factor
            fr[K::E + 36 + m] = cmk<C>(cv, sv);
        } else if (i == NB + Q::R0) {
            sincos_r(-al * (R)I.R0, &sv, &cv);
            fr[K::E + 16] = cmk<C>(cv, sv);      // x >= R0
            fr[K::E + 17] = cmk<C>(cv, -sv);     // x <= -R0
        } else {
            const int k = i - (NB + Q::R0 + 1);  // 0..15
            const int n = k < 8 ? I.iL + k : I.iR - 16 + k;
            sincos_r(-al * ((R)I.x0 + (R)n * (R)I.h), &sv, &cv);
            fr[K::E + 20 + k] = cmk<C>(cv, sv);
        }
    }
}

// Inverse pass 0; with V set, followed by the potential factor of the next
// step on every output: the full e^{-iU tau} off the strip block, the half
// factor on it (U = U0(z) + E(t + tau/2) x, Sec. II under Eq. SSFFT).
template <typename R, int LOGN, int LOGE, int LOGRM, typename TW>
__device__ __forceinline__ void inv_pass0_v(typename CT<R>::C* S, const TW* __restrict__ Ws,
                                            const typename VabT<R>::T* __restrict__ TV,
                                            const typename CT<R>::C* fr, R al, const Inst1D& I, int tid,
                                            bool V) {
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    using G = PassGeom<LOGN, LOGRM, 0>;
    constexpr int N = K::N;
    constexpr int LOGR = G::LOGR, RR = 1 << LOGR;
    constexpr int s = G::S;                    // = N / RR
    constexpr int NB = G::LOGR;
    const int nb = I.nb, blk0 = I.blk0, iL = I.iL, iR = I.iR;
    const bool fld = V && I.has_field;
    C ft; ft.x = 1; ft.y = 0;
    C fcR = ft, fcL = ft;
    if (fld) {
        R sv, cv; sincos_r(-al * ((R)I.x0 + (R)tid * (R)I.h), &sv, &cv);
        ft = cmk<C>(cv, sv);
        fcR = fr[K::E + 16];
        fcL = fr[K::E + 17];
    }
#pragma unroll 1
    for (int u = 0; u < K::E / RR; ++u) {
        const int off = tid + u * K::T;        // L = N: a single block
        const int sb = swz<C>(off);
        C v[RR];
        constexpr bool FULL = TwLay<TW>::template full<LOGN, LOGRM, 0>();
        TW tb[FULL ? RR - 1 : 4];
        if constexpr (s > 1)
            load_tw<TW, TwLay<TW>::template rows<LOGN, LOGRM, 0>(), s, true>(
                tb, Ws + TwLay<TW>::template toff<LOGN, LOGRM, 0>() + off);
        LoadInv<C, TW, RR, s, 0, FULL>::run(S, v, tb, sb, s > 1);
        dft_reg<C, RR, +1>(v);
        if (!V) {
            StoreNat<C, RR, s, 0>::run(S, v, sb);
            continue;
        }
        C fb = ft, fb2 = ft;
        if (fld) {
            fb = cmul(ft, fr[u]);
            fb2 = cmul(fb, fb);
        }
#pragma unroll
        for (int m = 0; m < RR; ++m) {
            const int n = off + m * s;
            C x = vmul(v[bitrev_c(m, LOGR)], __ldg(&TV[n]));
            if (fld) {
                // off the block exp(-2i alpha x_n) from the squared tables; on it
                // the half factor exp(-i alpha x_n), clamped beyond +-R0.  FP64
                // (pipe-bound) branches, so that only one factor is formed (a
                // warp diverges only where it straddles the block's edge); FP32
                // (issue-bound) forms both, branch-free, so that the table
                // loads of all m issue early.
                const bool inb = ((n - blk0) & (N - 1)) < nb;
                C f;
                if constexpr (sizeof(R) == 8) {
                    if (inb) {
                        const C fh = cmul(fb, fr[K::E + m]);
                        f = n >= iR ? fcR : (n < iL ? fcL : fh);
                    } else {
                        f = cmul(fb2, fr[K::E + 36 + m]);
                    }
                } else {
                    const C fh = cmul(fb, fr[K::E + m]);
                    const C ff = cmul(fb2, fr[K::E + 36 + m]);
                    const C fk = n >= iR ? fcR : (n < iL ? fcL : fh);
                    f = inb ? fk : ff;
                }
                x = cmul(x, f);
            }
            S[sb ^ swz<C>(m * s)] = x;
        }
    }
}

// exp(-i alpha x_n) computed directly (strip rows inside R0 that the table
// of field_setup does not cover; kept out of line: not taken for contours
// whose strip block ends next to R0)
template <typename R, typename C>
__device__ __noinline__ C field_direct(R al, double x0, double h, int n) {
    R sv, cv;
    sincos_r(-al * ((R)x0 + (R)n * (R)h), &sv, &cv);
    return cmk<C>(cv, sv);
}

// half field factor on strip row n: clamped beyond +-R0, else exp(-i alpha x_n)
template <typename R, typename C, int E>
__device__ __forceinline__ C strip_field(const C* fr, R al, const Inst1D& I, int n) {
    if (n >= I.iR) return fr[E + 16];
    if (n < I.iL) return fr[E + 17];
    if (n < I.iL + 8) return fr[E + 20 + (n - I.iL)];
    if (n >= I.iR - 8) return fr[E + 28 + (n - (I.iR - 8))];
    return field_direct<R, C>(al, I.x0, I.h, n);
}

// Sum of four complex values over the group; thread 0 writes them to out.
// scratch: 4 * (T/32) complex (the scan scratch, free at this point).
template <typename C, int T, class B>
__device__ __forceinline__ void surf_reduce(C (&acc)[4], C* scratch, int tid, B bar, C* __restrict__ out) {
    static_assert(T / 32 <= 16, "scratch of 64 complex");
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, o);
            acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, o);
        }
    if ((tid & 31) == 0)
#pragma unroll
        for (int r = 0; r < 4; ++r) scratch[4 * (tid >> 5) + r] = acc[r];
    bar.sync();
    if (tid == 0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            C t = cmk<C>(0, 0);
            for (int w = 0; w < (T + 31) / 32; ++w) t = cadd(t, scratch[4 * w + r]);
            out[r] = t;
        }
    }
}

// n 16-byte table entries from global to shared memory by nt threads
template <typename TT>
__device__ __forceinline__ void copy16(TT* dst, const TT* __restrict__ src, int n, int t, int nt) {
    static_assert(sizeof(TT) == 16, "16-byte entries");
    for (int i = t; i < n; i += nt)
        reinterpret_cast<float4*>(dst)[i] = __ldg(reinterpret_cast<const float4*>(src) + i);
}

// shared-memory bytes of one instance's private part: the state (unless
// GM), 64 complex of scan scratch and E + 52 field phases
template <typename R, int LOGN, int LOGE, int LOGRM>
__host__ __device__ constexpr size_t soft1d_inst_smem() {
    return sizeof(typename CT<R>::C) *
           ((Cfg1D<R, LOGN, LOGE, LOGRM>::GM ? 0 : (size_t(1) << LOGN)) + 64 + (size_t(1) << LOGE) + 52);
}

// All nsteps steps of one instance, run by the T threads of a group (tid =
// index in the group, bar = its barrier).  Ss: the state in shared memory
// (unused with GM); scan: 64 complex of scan scratch followed by E + 52
// field phases; Ws: the twiddle bases, already in shared memory and visible
// to the group by its first barrier.
//
// SURF: sample psi and psi' at the two surfaces into samples[0 ..
// nsteps][4] (soft1d_surf_kernel; sw holds two sets of four weight rows:
// for the state at the call's start and, with the half kinetic factor
// e^{-iK tau/2} folded in, for the state after each step).
template <typename R, int LOGN, int LOGE, int LOGRM, class B, bool SURF = false>
__device__ __forceinline__ void soft1d_run(const Inst1D& I, void* __restrict__ psi_base, int64_t nsteps,
                                           const double* __restrict__ ftab_base, int64_t ftab_stride,
                                           int* __restrict__ status, typename CT<R>::C* Ss,
                                           typename CT<R>::C* scan, const typename TwT<R>::T* Ws, int tid,
                                           B bar, const typename CT<R>::C* __restrict__ sw = nullptr,
                                           typename CT<R>::C* __restrict__ samples = nullptr)
{
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    constexpr int N = K::N, T = K::T, E = K::E;
    static_assert(K::NPASS >= 2, "at least two FFT passes");
    static_assert(Step1D<R, LOGN, LOGRM>::R0 <= 16, "pass radix <= 16");
    C* fr = scan + 64;               // E + 52 complex: field phases (field_setup)

    C* __restrict__ g_psi = reinterpret_cast<C*>(psi_base) + I.off;
    // the state: shared memory, or (GM) the instance's buffer itself
    C* S = K::GM ? g_psi : Ss;
    using TT = typename K::TT;
    const TT* __restrict__ TK = reinterpret_cast<const TT*>(I.TK);
    const TT* __restrict__ TKh = reinterpret_cast<const TT*>(I.TKh);
    using VT = typename VabT<R>::T;
    const VT* __restrict__ TV = reinterpret_cast<const VT*>(I.TV);
    const C* __restrict__ cn = reinterpret_cast<const C*>(I.cn);
    const VT* __restrict__ TVs = reinterpret_cast<const VT*>(I.TVs);
    const int nb = I.nb, blk0 = I.blk0;
    if (nsteps <= 0) return;

    // load the state (GM: permute the buffer into the swizzled order in place;
    // swz is an involution, so it is a product of disjoint swaps)
    if constexpr (K::GM) {
        for (int j = 0; j < E; ++j) {
            const int n = tid + j * T, p = swz<C>(n);
            if (n < p) { const C a = S[n]; S[n] = S[p]; S[p] = a; }
        }
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int n = tid + j * T;
            S[swz<C>(n)] = g_psi[n];
        }
    }
    bar.sync();

    const double* __restrict__ ftab = I.has_field ? ftab_base + (int64_t)I.fcls * ftab_stride : nullptr;
    // field amplitude of step s: alpha = tau E(t + tau/2) / 2
    auto alpha = [&](int64_t st) -> R { return (R)(0.5 * I.tau * I.E0 * __ldg(&ftab[st])); };

    // Pass step = -1 is the first half-kinetic factor of the call; every pass
    // ends with the potential factor of the next step, applied as the last
    // inverse FFT pass stores (none after the final half-kinetic factor).
    R al = 0;
    for (int64_t step = -1; step < nsteps; ++step) {
        // ---- Crank-Nicolson on the strip block, then the second e^{-iU tau/2}
        if (step >= 0 && nb > 0) {
            strip_cn_1d<C, VT, T, K::CMAX, N>(S, cn, TVs, nb, blk0, tid, scan, [&](int n, const VT& tv, C v) {
                v = vmul(v, tv);
                if (I.has_field) v = cmul(v, strip_field<R, C, E>(fr, al, I, n));
                return v;
            }, bar);
            bar.sync();
        }
        // ---- kinetic: forward FFT, e^{-iK tau} (e^{-iK tau/2} in the first
        //      and last pass of the call), inverse FFT, potential of the next step
        const bool more = step + 1 < nsteps;
        fwd_passes<R, LOGN, LOGE, LOGRM, 0, K::NPASS - 1>(S, Ws, tid, bar);
        if constexpr (SURF) {
            C acc[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[r] = cmk<C>(0, 0);
            kcenter<R, LOGN, LOGE, LOGRM, true>(S, (step >= 0 && more) ? TK : TKh, tid,
                                                sw + (step >= 0 ? 4 * N : 0), acc);
            surf_reduce<C, T>(acc, scan, tid, bar, samples + 4 * (step + 1));
        } else {
            kcenter<R, LOGN, LOGE, LOGRM>(S, (step >= 0 && more) ? TK : TKh, tid);
        }
        if (more && I.has_field) {
            al = alpha(step + 1);
            field_setup<R, LOGN, LOGE, LOGRM>(fr, al, I, tid);
        }
        bar.sync();
        inv_passes<R, LOGN, LOGE, LOGRM, K::NPASS - 2, 1>(S, Ws, tid, bar);
        inv_pass0_v<R, LOGN, LOGE, LOGRM>(S, Ws, TV, fr, al, I, tid, more);
        bar.sync();
    }

    // store
    if constexpr (K::GM) {
        for (int j = 0; j < E; ++j) {
            const int n = tid + j * T, p = swz<C>(n);
            if (n < p) { const C a = S[n]; S[n] = S[p]; S[p] = a; }
        }
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int n = tid + j * T;
            g_psi[n] = S[swz<C>(n)];
        }
    }
    if (tid == 0 && status) {
        const C v = S[0];
        if (!(isfinite((double)v.x) && isfinite((double)v.y))) atomicOr(status, 1);
    }
}

// One CTA per instance: blockIdx.x indexes insts.
template <typename R, int LOGN, int LOGE, int LOGRM>
__global__ void __launch_bounds__(Cfg1D<R, LOGN, LOGE, LOGRM>::T, Cfg1D<R, LOGN, LOGE, LOGRM>::MINB)
soft1d_kernel(const Inst1D* __restrict__ insts, void* __restrict__ psi_base, int64_t nsteps,
              const double* __restrict__ ftab_base, int64_t ftab_stride, int* __restrict__ status)
{
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using Q = Step1D<R, LOGN, LOGRM>;
    using C = typename K::C;
    static_assert(soft1d_smem<R, LOGN, LOGE, LOGRM>() <= 227 * 1024, "shared memory");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using TWT = typename TwT<R>::T;
    // layout: [state (unless GM)] [twiddles] [scan] [field phases]
    C* Ss = reinterpret_cast<C*>(smem_raw);
    TWT* Ws = reinterpret_cast<TWT*>(Ss + (K::GM ? 0 : K::N));
    const Inst1D I = insts[blockIdx.x];
    const TWT* __restrict__ W = reinterpret_cast<const TWT*>(I.W);
    if (nsteps <= 0) return;
    copy16(Ws, W, Q::TWN, threadIdx.x, K::T);
    // the run's first barrier (after its state load) also covers the twiddles
    soft1d_run<R, LOGN, LOGE, LOGRM>(I, psi_base, nsteps, ftab_base, ftab_stride, status, Ss,
                                     reinterpret_cast<C*>(Ws + Q::TWN), Ws, (int)threadIdx.x, BarCTA());
}

// One instance (blockIdx.x 0) with surface sampling: samples[s][r] for the
// state at the call's start plus s steps, rows psi(R), psi'(R), psi(-R),
// psi'(-R) (sw: the eight weight rows, see soft1d_run).
template <typename R, int LOGN, int LOGE, int LOGRM>
__global__ void __launch_bounds__(Cfg1D<R, LOGN, LOGE, LOGRM>::T, Cfg1D<R, LOGN, LOGE, LOGRM>::MINB)
soft1d_surf_kernel(const Inst1D* __restrict__ insts, void* __restrict__ psi_base, int64_t nsteps,
                   const double* __restrict__ ftab_base, int64_t ftab_stride, int* __restrict__ status,
                   const void* __restrict__ sw, void* __restrict__ samples)
{
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using Q = Step1D<R, LOGN, LOGRM>;
    using C = typename K::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using TWT = typename TwT<R>::T;
    C* Ss = reinterpret_cast<C*>(smem_raw);
    TWT* Ws = reinterpret_cast<TWT*>(Ss + (K::GM ? 0 : K::N));
    const Inst1D I = insts[0];
    const TWT* __restrict__ W = reinterpret_cast<const TWT*>(I.W);
    if (nsteps <= 0) return;
    copy16(Ws, W, Q::TWN, threadIdx.x, K::T);
    soft1d_run<R, LOGN, LOGE, LOGRM, BarCTA, true>(I, psi_base, nsteps, ftab_base, ftab_stride, status, Ss,
                                                   reinterpret_cast<C*>(Ws + Q::TWN), Ws, (int)threadIdx.x,
                                                   BarCTA(), reinterpret_cast<const C*>(sw),
                                                   reinterpret_cast<C*>(samples));
}

template <typename R, int LOGN, int LOGE, int LOGRM>
int launch_soft1d_surf_t(const Inst1D* d_inst, void* psi, int64_t nsteps, const double* ftab, int64_t ftab_stride,
                         int* d_status, const void* sw, void* samples, cudaStream_t st)
{
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    auto kern = soft1d_surf_kernel<R, LOGN, LOGE, LOGRM>;
    const size_t smem = soft1d_smem<R, LOGN, LOGE, LOGRM>();
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SOFT_ERR_CUDA;
    kern<<<1, K::T, smem, st>>>(d_inst, psi, nsteps, ftab, ftab_stride, d_status, sw, samples);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

template <typename R, int LOGN, int LOGE, int LOGRM>
int launch_soft1d_t(const Inst1D* d_inst, int count, void* psi, int64_t nsteps,
                    const double* ftab, int64_t ftab_stride, int* d_status, cudaStream_t st,
                    size_t* smem_out)
{
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    auto kern = soft1d_kernel<R, LOGN, LOGE, LOGRM>;
    const size_t smem = soft1d_smem<R, LOGN, LOGE, LOGRM>();
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
