// Device helpers shared by the kernels of this library: complex arithmetic on
// float2/double2, shared-memory swizzles, in-register radix-2^k DFTs and a
// block-wide scan of affine maps (used by the strip Crank-Nicolson solve).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace soft {

// Barrier of the threads that own one transform: the whole CTA
// (__syncthreads), or one warp-aligned group of a CTA that runs several
// transforms side by side (named barrier `id`, `n` threads).
struct BarCTA {
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct BarGroup {
    int id, n;
    __device__ __forceinline__ void sync() const {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
    }
};

// Asynchronous global -> shared copies of 8 or 16 bytes (cp.async): the
// copies of a thread are in flight together with no register staging;
// cp_async_wait<0>() waits for the thread's own copies (a barrier after it
// publishes them to the other threads).  Both addresses must be aligned to
// the copy size.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    static_assert(BYTES == 8 || BYTES == 16, "8- or 16-byte copies");
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename R> struct CT;
template <> struct CT<float> { using C = float2; };
template <> struct CT<double> { using C = double2; };

template <typename C> __device__ __forceinline__ C cmk(decltype(C::x) x, decltype(C::x) y) {
    C c; c.x = x; c.y = y; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
    return cmk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// a*b + c
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C c) {
    return cmk<C>(c.x + a.x * b.x - a.y * b.y, c.y + a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) {
    return cmk<C>(a.x * s, a.y * s);
}

// XOR swizzle of a shared-memory complex array: 128-byte rows, the column
// index is XORed with the row index so that strided butterfly accesses of
// every stride spread over all banks.  The map is linear over XOR, so for a
// butterfly whose element offsets j*s share no bits with its base,
// swz(base + j*s) = swz(base) ^ swz(j*s) with the second term a constant.
template <typename C> __host__ __device__ __forceinline__ constexpr int swz(int i) {
    return sizeof(C) == 8 ? (i ^ ((i >> 4) & 15)) : (i ^ ((i >> 3) & 7));
}

// ---------------------------------------------------------------------------
// In-register DFT of R = 2^k points, y_m = sum_j v_j exp(SIGN 2 pi i j m / R),
// computed by a decimation-in-frequency radix-2 network: natural order in,
// bit-reversed order out (y_m ends in v[bitrev(m)]).
__host__ __device__ constexpr int bitrev_c(int x, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}

// cos(2 pi t / 16) and sin(2 pi t / 16) for t = 0..15
__host__ __device__ constexpr double cos16(int t) {
    constexpr double c[16] = {1.0, 0.92387953251128674, 0.70710678118654752, 0.38268343236508977,
                              0.0, -0.38268343236508977, -0.70710678118654752, -0.92387953251128674,
                              -1.0, -0.92387953251128674, -0.70710678118654752, -0.38268343236508977,
                              0.0, 0.38268343236508977, 0.70710678118654752, 0.92387953251128674};
    return c[t & 15];
}
__host__ __device__ constexpr double sin16(int t) { return cos16(t - 4); }

// FP32 split of an FP64 constant v = hi + lo (|lo| <= ulp(hi)/2)
__host__ __device__ constexpr float f32_hi(double v) { return (float)v; }
__host__ __device__ constexpr float f32_lo(double v) { return (float)(v - (double)(float)v); }

// multiply by exp(SIGN 2 pi i t / R) with t, R compile-time.
// FP32: every rounded (cos, sin) pair of an angle k pi/8 that is not a
// multiple of pi/2 has a modulus below 1 (|w|^2 - 1 = -3.4e-8 at pi/4 and
// -5.7e-8 at odd multiples of pi/8).  Applied to the same positions of every
// butterfly, in each pass of the forward and the inverse FFT, that is a
// coherent loss of about 1e-7 per time step which grows linearly over a
// propagation.  The constants are therefore applied as FP32 hi + lo pairs
// (modulus exact to ~2^-48); only the data-dependent roundings remain.
template <typename C, int R, int SIGN, int t>
__device__ __forceinline__ C twc(C a) {
    using F = decltype(C::x);
    constexpr int t16 = (t * 16 / R) & 15;   // same angle in 16ths
    if constexpr (t16 == 0) {
        return a;
    } else if constexpr (t16 == 4) {           // exp(SIGN i pi/2) = SIGN i
        return SIGN > 0 ? cmk<C>(-a.y, a.x) : cmk<C>(a.y, -a.x);
    } else if constexpr (t16 == 8) {
        return cmk<C>(-a.x, -a.y);
    } else if constexpr (t16 == 12) {
        return SIGN > 0 ? cmk<C>(a.y, -a.x) : cmk<C>(-a.y, a.x);
    } else if constexpr (sizeof(F) == 4 && (t16 & 3) == 2) {
        // |cos| = |sin| = 1/sqrt(2): re = r (sc a.x - ss a.y), im = r (ss a.x + sc a.y)
        constexpr double cd = cos16(t16), sd = SIGN * sin16(t16);
        constexpr double r = 0.70710678118654752440;
        constexpr float rh = f32_hi(r), rl = f32_lo(r);
        const float u = (cd > 0 ? a.x : -a.x) - (sd > 0 ? a.y : -a.y);
        const float v = (sd > 0 ? a.x : -a.x) + (cd > 0 ? a.y : -a.y);
        return cmk<C>(fmaf(u, rh, u * rl), fmaf(v, rh, v * rl));
    } else if constexpr (sizeof(F) == 4) {
        constexpr double cd = cos16(t16), sd = SIGN * sin16(t16);
        constexpr float ch = f32_hi(cd), cl = f32_lo(cd), sh = f32_hi(sd), sl = f32_lo(sd);
        return cmk<C>(fmaf(a.x, ch, fmaf(-a.y, sh, fmaf(a.x, cl, -a.y * sl))),
                      fmaf(a.x, sh, fmaf(a.y, ch, fmaf(a.x, sl, a.y * cl))));
    } else {
        constexpr F c = (F)cos16(t16);
        constexpr F s = (F)(SIGN * sin16(t16));
        return cmk<C>(a.x * c - a.y * s, a.x * s + a.y * c);
    }
}

template <typename C, int R, int SIGN, int SPAN, int BLK, int J>
__device__ __forceinline__ void dif_bfly(C* v) {
    C a = v[BLK + J], b = v[BLK + J + SPAN];
    v[BLK + J] = cadd(a, b);
    v[BLK + J + SPAN] = twc<C, 2 * SPAN, SIGN, J>(csub(a, b));
}

template <typename C, int R, int SIGN, int SPAN, int BLK, int J>
struct DifJ {
    __device__ __forceinline__ static void run(C* v) {
        dif_bfly<C, R, SIGN, SPAN, BLK, J>(v);
        if constexpr (J + 1 < SPAN) DifJ<C, R, SIGN, SPAN, BLK, J + 1>::run(v);
    }
};
template <typename C, int R, int SIGN, int SPAN, int BLK>
struct DifBlk {
    __device__ __forceinline__ static void run(C* v) {
        DifJ<C, R, SIGN, SPAN, BLK, 0>::run(v);
        if constexpr (BLK + 2 * SPAN < R) DifBlk<C, R, SIGN, SPAN, BLK + 2 * SPAN>::run(v);
    }
};
template <typename C, int R, int SIGN, int SPAN>
struct DifStage {
    __device__ __forceinline__ static void run(C* v) {
        DifBlk<C, R, SIGN, SPAN, 0>::run(v);
        if constexpr (SPAN > 1) DifStage<C, R, SIGN, SPAN / 2>::run(v);
    }
};

template <typename C, int R, int SIGN>
__device__ __forceinline__ void dft_reg(C* v) {
    if constexpr (R > 1) DifStage<C, R, SIGN, R / 2>::run(v);
}

// ---------------------------------------------------------------------------
// Block-wide scan of affine maps f(y) = M y + Y (complex), composed in thread
// order (REV = false: thread 0 first; REV = true: thread T-1 first).  Returns,
// for each thread, the value produced by all preceding maps applied to 0, i.e.
// the carry that enters this thread's chunk.  scratch: 2 * (T/32) complex.
// tid is the thread's index in the group of T threads (warp-aligned) that
// runs the scan, bar that group's barrier.
template <typename C, int T, bool REV, class B = BarCTA>
__device__ __forceinline__ C affine_carry(C M, C Y, C* scratch, int tid = -1, B bar = B()) {
    if (tid < 0) tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int NW = T / 32;
    // inclusive warp scan
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        C Mo, Yo;
        if constexpr (!REV) {
            Mo.x = __shfl_up_sync(0xffffffffu, M.x, d); Mo.y = __shfl_up_sync(0xffffffffu, M.y, d);
            Yo.x = __shfl_up_sync(0xffffffffu, Y.x, d); Yo.y = __shfl_up_sync(0xffffffffu, Y.y, d);
            if (lane >= d) { Y = cfma(M, Yo, Y); M = cmul(M, Mo); }
        } else {
            Mo.x = __shfl_down_sync(0xffffffffu, M.x, d); Mo.y = __shfl_down_sync(0xffffffffu, M.y, d);
            Yo.x = __shfl_down_sync(0xffffffffu, Y.x, d); Yo.y = __shfl_down_sync(0xffffffffu, Y.y, d);
            if (lane + d < 32) { Y = cfma(M, Yo, Y); M = cmul(M, Mo); }
        }
    }
    // exclusive within the warp: value of the preceding lane
    C Yex;
    if constexpr (!REV) {
        Yex.x = __shfl_up_sync(0xffffffffu, Y.x, 1); Yex.y = __shfl_up_sync(0xffffffffu, Y.y, 1);
        if (lane == 0) { Yex.x = 0; Yex.y = 0; }
    } else {
        Yex.x = __shfl_down_sync(0xffffffffu, Y.x, 1); Yex.y = __shfl_down_sync(0xffffffffu, Y.y, 1);
        if (lane == 31) { Yex.x = 0; Yex.y = 0; }
    }
    // lane product for combining with earlier warps: the exclusive M
    C Mex;
    if constexpr (!REV) {
        Mex.x = __shfl_up_sync(0xffffffffu, M.x, 1); Mex.y = __shfl_up_sync(0xffffffffu, M.y, 1);
        if (lane == 0) { Mex.x = 1; Mex.y = 0; }
    } else {
        Mex.x = __shfl_down_sync(0xffffffffu, M.x, 1); Mex.y = __shfl_down_sync(0xffffffffu, M.y, 1);
        if (lane == 31) { Mex.x = 1; Mex.y = 0; }
    }
    if constexpr (NW == 1) {
        return Yex;
    } else {
        const int tail = REV ? 0 : 31;
        if (lane == tail) { scratch[2 * warp] = M; scratch[2 * warp + 1] = Y; }
        bar.sync();
        // carry entering each warp: warp 0 scans the warp totals (lane l holds
        // the l-th warp in composition order) and leaves warp w's carry in
        // scratch[2 w]
        if (warp == 0) {
            const int w = REV ? NW - 1 - lane : lane;
            C Mw, Yw;
            Mw.x = 1; Mw.y = 0; Yw.x = 0; Yw.y = 0;
            if (lane < NW) { Mw = scratch[2 * w]; Yw = scratch[2 * w + 1]; }
#pragma unroll
            for (int d = 1; d < NW; d <<= 1) {
                C Mo, Yo;
                Mo.x = __shfl_up_sync(0xffffffffu, Mw.x, d); Mo.y = __shfl_up_sync(0xffffffffu, Mw.y, d);
                Yo.x = __shfl_up_sync(0xffffffffu, Yw.x, d); Yo.y = __shfl_up_sync(0xffffffffu, Yw.y, d);
                if (lane >= d) { Yw = cfma(Mw, Yo, Yw); Mw = cmul(Mw, Mo); }
            }
            C cw;
            cw.x = __shfl_up_sync(0xffffffffu, Yw.x, 1); cw.y = __shfl_up_sync(0xffffffffu, Yw.y, 1);
            if (lane == 0) { cw.x = 0; cw.y = 0; }
            __syncwarp();
            if (lane < NW) scratch[2 * w] = cw;
        }
        bar.sync();
        const C carry = scratch[2 * warp];
        bar.sync();
        return cfma(Mex, carry, Yex);
    }
}

}  // namespace soft
