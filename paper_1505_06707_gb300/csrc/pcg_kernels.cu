// Complex-symmetric CG (Sec. III) for the 2D stationary ECS equation:
// instantiations of the A-apply and preconditioner passes and the vector /
// scalar kernels of the iteration.
//
// Pass precisions (compute R, vector I/O IO):
//   FP64 path (precond 0, 1)          A and P^-1: R double, IO complex128
//   FP32 preconditioner (precond 4)   P^-1: R float, IO complex128
//   mixed iteration (precond 5)       A and P^-1: R float, IO complex64; the
//                                     energies that fall back: A with R double,
//                                     IO complex64
#include "pcg.cuh"
#include "pcg_launch.h"

namespace soft {

namespace {

constexpr int TWP = 2;    // columns per CTA of the FP64 column passes
// columns per CTA of the FP32 column passes: 8 (64-byte row runs of
// complex64), fewer where that would exceed 1024 threads
template <int LN>
struct Tw32 {
    static constexpr int T = Cfg1D<float, LN, 3, 3>::T;
    static constexpr int value = 1024 / T < 8 ? 1024 / T : 8;
};

// CTAs per SM: 1024 threads per SM, <= 64 registers (FP32 column passes)
template <int THREADS>
struct MinB32 { static constexpr int value = THREADS >= 1024 ? 1 : 1024 / THREADS; };

inline int done() { return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA; }

template <class Kern>
inline bool set_smem(Kern k, size_t smem) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess;
}

template <typename R, typename IO, int LN, int LE, int LR>
int a_row(const PcgGeo& g, const void* p, void* w, const double* E, const int* act, int nE,
          cudaStream_t st) {
    using K = Cfg1D<R, LN, LE, LR>;
    const size_t smem = sizeof(typename K::C) * 2 * K::N + 64;
    auto k = a_row_kernel<R, IO, LN, LE, LR>;
    if (!set_smem(k, smem)) return SOFT_ERR_CUDA;
    if (nE > 0) k<<<dim3(g.ny, nE), K::T, smem, st>>>(g, p, w, E, act);
    return done();
}

template <typename R, typename IO, int LN, int LE, int LR, int TW, int MB>
int a_col(const PcgGeo& g, const void* p, void* w, const int* act, double2* part, int pstride, int nE,
          cudaStream_t st) {
    using K = Cfg1D<R, LN, LE, LR>;
    using C = typename K::C;
    const size_t smem = sizeof(C) * 2 * TW * ColPitch<C, K::N>::value + 64;
    auto k = a_col_kernel<R, IO, LN, LE, LR, TW, MB>;
    if (!set_smem(k, smem)) return SOFT_ERR_CUDA;
    const int nb = g.nx / TW;
    if (nE > 0) k<<<dim3(nb, nE), TW * K::T, smem, st>>>(g, p, w, act, part, pstride > nb ? pstride : nb);
    return done();
}

// which 1: t = X_x F_x a; which 2: b = F_x^-1 X_x^T a, partials r^T b, b^T w
template <typename R, typename IO, int LN, int LE, int LR>
int pc_row(int which, const PcgGeo& g, const void* a, void* b, const void* r, const void* w, const int* act,
           double2* part, double2* part2, int nE, cudaStream_t st) {
    using K = Cfg1D<R, LN, LE, LR>;
    const size_t smem = sizeof(typename K::C) * 2 * K::N + 64;
    const dim3 grid(g.ny, nE);
    if (which == 1) {
        auto k = pc_row1_kernel<R, IO, LN, LE, LR>;
        if (!set_smem(k, smem)) return SOFT_ERR_CUDA;
        if (nE > 0) k<<<grid, K::T, smem, st>>>(g, a, b, act);
    } else {
        auto k = pc_row2_kernel<R, IO, LN, LE, LR>;
        if (!set_smem(k, smem)) return SOFT_ERR_CUDA;
        if (nE > 0) k<<<grid, K::T, smem, st>>>(g, a, b, r, w, act, part, part2);
    }
    return done();
}

template <typename R, int LN, int LE, int LR, int TW, int MB>
int pc_col(const PcgGeo& g, void* t, const double* E, const int* act, int nE, cudaStream_t st) {
    using K = Cfg1D<R, LN, LE, LR>;
    using C = typename K::C;
    const size_t smem = sizeof(C) * 2 * TW * ColPitch<C, K::N>::value + 64;
    auto k = pc_col_kernel<R, LN, LE, LR, TW, MB>;
    if (!set_smem(k, smem)) return SOFT_ERR_CUDA;
    if (nE > 0) k<<<dim3(g.nx / TW, nE), TW * K::T, smem, st>>>(g, t, E, act);
    return done();
}

}  // namespace

// every pass runs with LOGE = LOGRM = 3 (radix 8, eight elements per thread)
#define PCG_SIZES(CALL)                                  \
    switch (logn) {                                      \
    case 8: return CALL(8);                              \
    case 9: return CALL(9);                              \
    case 10: return CALL(10);                            \
    case 11: return CALL(11);                            \
    }                                                    \
    return SOFT_ERR_UNSUPPORTED;

int pcg_row(int logn, int which, const PcgGeo& g, const void* a, void* b, const void* c,
            const double* E, const int* act, double2* part, int nE, cudaStream_t st) {
#define CALL(L) (which == 0 ? a_row<double, double2, L, 3, 3>(g, a, b, E, act, nE, st) \
                            : pc_row<double, double2, L, 3, 3>(which, g, a, b, c, nullptr, act, part, nullptr, nE, st))
    PCG_SIZES(CALL)
#undef CALL
}

int pcg_col(int logn, int which, const PcgGeo& g, const void* a, void* b, const double* E,
            const int* act, double2* part, int nE, cudaStream_t st) {
#define CALL(L) (which == 0 ? a_col<double, double2, L, 3, 3, TWP, 1>(g, a, b, act, part, 0, nE, st) \
                            : pc_col<double, L, 3, 3, TWP, 1>(g, b, E, act, nE, st))
    PCG_SIZES(CALL)
#undef CALL
}

int pcg_col_blocks(int nx) { return nx / TWP; }

int pcg_pc32_row(int logn, int which, const PcgGeo& g, const void* a, void* b, const void* c,
                 const int* act, double2* part, int nE, cudaStream_t st) {
#define CALL(L) pc_row<float, double2, L, 3, 3>(which, g, a, b, c, nullptr, act, part, nullptr, nE, st)
    PCG_SIZES(CALL)
#undef CALL
}

int pcg_pc32_col(int logn, const PcgGeo& g, void* b, const double* E, const int* act, int nE,
                 cudaStream_t st) {
#define CALL(L) pc_col<float, L, 3, 3, Tw32<L>::value, MinB32<Tw32<L>::value * Tw32<L>::T>::value>(g, b, E, act, nE, st)
    PCG_SIZES(CALL)
#undef CALL
}

int pcg_pc32f_row(int logn, int which, const PcgGeo& g, const void* a, void* b, const void* r, const void* w,
                  const int* act, double2* part, double2* part2, int nE, cudaStream_t st) {
#define CALL(L) pc_row<float, float2, L, 3, 3>(which, g, a, b, r, w, act, part, part2, nE, st)
    PCG_SIZES(CALL)
#undef CALL
}

int pcg_a32_row(int logn, const PcgGeo& g, const void* p, void* w, const double* E, const int* act,
                int nE, cudaStream_t st) {
#define CALL(L) a_row<float, float2, L, 3, 3>(g, p, w, E, act, nE, st)
    PCG_SIZES(CALL)
#undef CALL
}

int pcg_a32_col(int logn, const PcgGeo& g, const void* p, void* w, const int* act, double2* part,
                int pstride, int nE, cudaStream_t st) {
#define CALL(L) a_col<float, float2, L, 3, 3, Tw32<L>::value, MinB32<Tw32<L>::value * Tw32<L>::T>::value>( \
    g, p, w, act, part, pstride, nE, st)
    PCG_SIZES(CALL)
#undef CALL
}

int pcg_a64f_row(int logn, const PcgGeo& g, const void* p, void* w, const double* E, const int* act,
                 int nE, cudaStream_t st) {
#define CALL(L) a_row<double, float2, L, 3, 3>(g, p, w, E, act, nE, st)
    PCG_SIZES(CALL)
#undef CALL
}

int pcg_a64f_col(int logn, const PcgGeo& g, const void* p, void* w, const int* act, double2* part,
                 int pstride, int nE, cudaStream_t st) {
#define CALL(L) a_col<double, float2, L, 3, 3, TWP, 1>(g, p, w, act, part, pstride, nE, st)
    PCG_SIZES(CALL)
#undef CALL
}
#undef PCG_SIZES


// ------------------------------------------------------------ vector kernels
__device__ __forceinline__ double2 sum_warp(double2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// x = 0, r = f for every energy
__global__ void vec_init_kernel(const double2* __restrict__ f, double2* __restrict__ x,
                                double2* __restrict__ r, int64_t N, int nE) {
    const int64_t tot = N * nE;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = make_double2(0.0, 0.0);
        r[i] = f[i % N];
    }
}

// partial sums of |f|^2 (one vector)
__global__ void vec_norm2_kernel(const double2* __restrict__ f, int64_t N, double2* __restrict__ part) {
    __shared__ double2 red[32];
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = f[i];
        acc.x += v.x * v.x + v.y * v.y;
    }
    const double2 t = block_sum2(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// x += alpha p, r -= alpha w; partial ||r||^2 per CTA
__global__ void vec_xr_kernel(double2* __restrict__ x, double2* __restrict__ r,
                              const double2* __restrict__ p, const double2* __restrict__ w,
                              const double2* __restrict__ alpha, const int* __restrict__ active,
                              int64_t N, double2* __restrict__ part) {
    const int e = blockIdx.y;
    if (!active[e]) return;
    __shared__ double2 red[32];
    const double2 a = alpha[e];
    const int64_t o = (int64_t)e * N;
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 pv = p[o + i], wv = w[o + i];
        double2 xv = x[o + i], rv = r[o + i];
        xv.x += a.x * pv.x - a.y * pv.y; xv.y += a.x * pv.y + a.y * pv.x;
        rv.x -= a.x * wv.x - a.y * wv.y; rv.y -= a.x * wv.y + a.y * wv.x;
        x[o + i] = xv;
        r[o + i] = rv;
        acc.x += rv.x * rv.x + rv.y * rv.y;
    }
    const double2 t = block_sum2(acc, red);
    if (threadIdx.x == 0) part[(int64_t)e * gridDim.x + blockIdx.x] = t;
}

// r = f - t for the energies with active set
__global__ void vec_sub_kernel(const double2* __restrict__ f, const double2* __restrict__ t,
                               double2* __restrict__ r, const int* __restrict__ active, int64_t N) {
    const int e = blockIdx.y;
    if (!active[e]) return;
    const int64_t o = (int64_t)e * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 fv = f[i], tv = t[o + i];
        r[o + i] = make_double2(fv.x - tv.x, fv.y - tv.y);
    }
}

// p = z + beta p (beta = 0 with copy = 1: p = z)
__global__ void vec_p_kernel(double2* __restrict__ p, const double2* __restrict__ z,
                             const double2* __restrict__ beta, const int* __restrict__ active,
                             int64_t N, int copy) {
    const int e = blockIdx.y;
    if (!active[e]) return;
    const double2 b = copy ? make_double2(0.0, 0.0) : beta[e];
    const int64_t o = (int64_t)e * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 zv = z[o + i];
        double2 pv = copy ? make_double2(0.0, 0.0) : p[o + i];
        p[o + i] = make_double2(zv.x + b.x * pv.x - b.y * pv.y, zv.y + b.x * pv.y + b.y * pv.x);
    }
}

// an energy leaves the iteration with status st
__device__ __forceinline__ void retire(const PcgState& s, int e, int st) {
    s.status[e] = st;
    s.active[e] = 0;
    if (s.act32) { s.act32[e] = 0; s.act64[e] = 0; }
    atomicSub(s.nactive, 1);
}

// sum of n partials by one warp: lane l adds l, l + 32, ... in order, then a
// fixed butterfly; every lane returns the total (same order on every call)
__device__ __forceinline__ double2 warp_sum_parts(const double2* __restrict__ p, int n) {
    double2 t = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < n; i += 32) { t.x += p[i].x; t.y += p[i].y; }
    return sum_warp(t);
}

// per-energy scalar updates of the iteration (one warp per energy; the
// partial sums are added in a fixed order, so results are reproducible)
__global__ void pcg_scalar_kernel(int stage, int nE, const double2* __restrict__ part, int nparts,
                                  PcgState s, const double2* __restrict__ part2) {
    const int e = blockIdx.x;
    if (stage == STAGE_FNORM) {
        if (e == 0) {
            const double2 t = warp_sum_parts(part, nparts);
            if (threadIdx.x == 0) *s.fnorm2 = t.x;
        }
        return;
    }
    if (e >= nE || !s.active[e]) return;
    if (stage == STAGE_TRUE && !s.upd[e]) return;
    const double2 t = warp_sum_parts(part + (int64_t)e * nparts, nparts);
    const double2 u = stage == STAGE_BETA_FLEX ? warp_sum_parts(part2 + (int64_t)e * nparts, nparts)
                                               : make_double2(0.0, 0.0);
    if (threadIdx.x != 0) return;
    if (stage == STAGE_RHO) {
        s.rho[e] = t;
        if (!(fabs(t.x) + fabs(t.y) > 1e-300)) { retire(s, e, SOFT_ERR_BREAKDOWN); }
    } else if (stage == STAGE_ALPHA) {
        const double d = t.x * t.x + t.y * t.y;
        if (!(d > 0.0) || !isfinite(d)) { retire(s, e, SOFT_ERR_BREAKDOWN); return; }
        const double2 rho = s.rho[e];                      // alpha = rho / (p^T w)
        s.alpha[e] = make_double2((rho.x * t.x + rho.y * t.y) / d, (rho.y * t.x - rho.x * t.y) / d);
    } else if (stage == STAGE_RNORM) {
        const double rel = sqrt(t.x / *s.fnorm2);
        s.relres[e] = rel;
        s.iters[e] += 1;
        if (!isfinite(rel)) { retire(s, e, SOFT_ERR_NONFINITE); }
        else if (rel < s.tol) { retire(s, e, SOFT_OK); }
    } else if (stage == STAGE_RNORM_RU) {
        // recursive residual of the FP32-A iteration: flag a true-residual
        // update once it has dropped by delta since the last one (or below tol)
        const double rel = sqrt(t.x / *s.fnorm2);
        s.relres[e] = rel;
        s.iters[e] += 1;
        s.upd[e] = 0;
        if (!isfinite(rel)) { retire(s, e, SOFT_ERR_NONFINITE); }
        else if (rel < fmax(s.tol, s.delta * s.rref[e]) || s.iters[e] - s.lastu[e] >= s.maxgap) s.upd[e] = 1;
    } else if (stage == STAGE_TRUE) {
        // true residual f - A x (A in FP64) replaces the recursive one; only
        // it decides convergence.  If it has not halved since the last update
        // (while the recursive one dropped by delta, or maxgap iterations
        // passed), the FP32 A no longer drives this energy's iteration: A is
        // applied in FP64 for it from here on, after a restart.
        const double rel = sqrt(t.x / *s.fnorm2);
        s.relres[e] = rel;
        s.upd[e] = 0;
        s.lastu[e] = s.iters[e];
        if (!isfinite(rel)) { retire(s, e, SOFT_ERR_NONFINITE); return; }
        if (rel < s.tol) { retire(s, e, SOFT_OK); return; }
        if (!(rel < 0.5 * s.rref[e])) {
            if (s.mode[e] & 1) {                           // stalled on the FP64 A too: leave the
                s.mode[e] |= 4;                            // mixed iteration for an FP64 restart
                retire(s, e, SOFT_ERR_NOT_CONVERGED);
                return;
            }
            s.mode[e] = 3;
            s.act32[e] = 0;
            s.act64[e] = 1;
        }
        s.rref[e] = rel;
    } else if (stage == STAGE_BETA_FLEX) {
        // flexible (Polak-Ribiere) beta = z'^T (r' - r) / rho = -alpha z'^T w / rho
        const double2 rho = s.rho[e], al = s.alpha[e];
        const double d = rho.x * rho.x + rho.y * rho.y;
        if (!(d > 0.0)) { retire(s, e, SOFT_ERR_BREAKDOWN); return; }
        const double2 au = make_double2(al.x * u.x - al.y * u.y, al.x * u.y + al.y * u.x);
        if (s.mode && (s.mode[e] & 2)) {                   // restart: p = z
            s.mode[e] &= ~2;
            s.beta[e] = make_double2(0.0, 0.0);
            s.rho[e] = t;
            return;
        }
        s.beta[e] = make_double2(-(au.x * rho.x + au.y * rho.y) / d, -(au.y * rho.x - au.x * rho.y) / d);
        s.rho[e] = t;
    } else if (stage == STAGE_BETA) {
        const double2 rho = s.rho[e];
        const double d = rho.x * rho.x + rho.y * rho.y;
        if (!(d > 0.0)) { retire(s, e, SOFT_ERR_BREAKDOWN); return; }
        s.beta[e] = make_double2((t.x * rho.x + t.y * rho.y) / d, (t.y * rho.x - t.x * rho.y) / d);
        s.rho[e] = t;
    }
}

int vec_init(const void* f, void* x, void* r, int64_t N, int nE, cudaStream_t st) {
    vec_init_kernel<<<1024, 256, 0, st>>>((const double2*)f, (double2*)x, (double2*)r, N, nE);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}
int vec_norm2(const void* f, int64_t N, double2* part, int nparts, cudaStream_t st) {
    vec_norm2_kernel<<<nparts, 256, 0, st>>>((const double2*)f, N, part);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}
int vec_xr(void* x, void* r, const void* p, const void* w, const double2* alpha, const int* act,
           int64_t N, int nE, double2* part, int nparts, cudaStream_t st) {
    vec_xr_kernel<<<dim3(nparts, nE), 256, 0, st>>>((double2*)x, (double2*)r, (const double2*)p,
                                                     (const double2*)w, alpha, act, N, part);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}
int vec_sub(const void* f, const void* t, void* r, const int* act, int64_t N, int nE, cudaStream_t st) {
    vec_sub_kernel<<<dim3(256, nE), 256, 0, st>>>((const double2*)f, (const double2*)t, (double2*)r, act, N);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}
int vec_p(void* p, const void* z, const double2* beta, const int* act, int64_t N, int nE, int copy,
          cudaStream_t st) {
    vec_p_kernel<<<dim3(256, nE), 256, 0, st>>>((double2*)p, (const double2*)z, beta, act, N, copy);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}
// r^T z and z^T w partials per CTA
__global__ void vec_dot2_kernel(const double2* __restrict__ r, const double2* __restrict__ z,
                                const double2* __restrict__ w, const int* __restrict__ active,
                                int64_t N, double2* __restrict__ p1, double2* __restrict__ p2) {
    const int e = blockIdx.y;
    if (!active[e]) return;
    __shared__ double2 red[32];
    const int64_t o = (int64_t)e * N;
    double2 a1 = make_double2(0.0, 0.0), a2 = make_double2(0.0, 0.0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 rv = r[o + i], zv = z[o + i], wv = w[o + i];
        a1.x += rv.x * zv.x - rv.y * zv.y; a1.y += rv.x * zv.y + rv.y * zv.x;
        a2.x += zv.x * wv.x - zv.y * wv.y; a2.y += zv.x * wv.y + zv.y * wv.x;
    }
    const double2 t1 = block_sum2(a1, red);
    if (threadIdx.x == 0) p1[(int64_t)e * gridDim.x + blockIdx.x] = t1;
    const double2 t2 = block_sum2(a2, red);
    if (threadIdx.x == 0) p2[(int64_t)e * gridDim.x + blockIdx.x] = t2;
}

int vec_dot2(const void* r, const void* z, const void* w, const int* act, int64_t N, int nE,
             double2* part1, double2* part2, int nparts, cudaStream_t st) {
    vec_dot2_kernel<<<dim3(nparts, nE), 256, 0, st>>>((const double2*)r, (const double2*)z,
                                                       (const double2*)w, act, N, part1, part2);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

// -------------------------------------- mixed iteration (complex64 vectors)
// r, p, z, w are complex64; the solution increment since the last true-
// residual update is a double-float pair (xh + xl, about 48 significant
// bits), folded into the complex128 x at each update.  Double-float sums use
// Knuth's TwoSum and Dekker's Fast2Sum, products the FMA-based TwoProduct.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {   // |a| >= |b|
    s = a + b;
    e = b - (s - a);
}
// (xh, xl) += (yh, yl)
__device__ __forceinline__ void df_add(float& xh, float& xl, float yh, float yl) {
    float s, e;
    two_sum(xh, yh, s, e);
    e += xl + yl;
    fast_two_sum(s, e, xh, xl);
}
// (ah + al) b as an unnormalised pair (ph, pl)
__device__ __forceinline__ void df_mul(float ah, float al, float b, float& ph, float& pl) {
    ph = ah * b;
    pl = fmaf(ah, b, -ph);
    pl = fmaf(al, b, pl);
}
__device__ __forceinline__ void df_split(double a, float& h, float& l) {
    h = (float)a;
    l = (float)(a - (double)h);
}

// x = 0, r = f (rounded), increment = 0
__global__ void vec_init32_kernel(const double2* __restrict__ f, double2* __restrict__ x, float2* __restrict__ r,
                                  float2* __restrict__ xh, float2* __restrict__ xl, int64_t N, int nE) {
    const int64_t tot = N * nE;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 fv = f[i % N];
        x[i] = make_double2(0.0, 0.0);
        r[i] = make_float2((float)fv.x, (float)fv.y);
        xh[i] = make_float2(0.f, 0.f);
        xl[i] = make_float2(0.f, 0.f);
    }
}

// increment += alpha p (double-float), r -= alpha w (FP32); partial ||r||^2
// (each thread sums its terms in FP32, the block sum is FP64)
__global__ void vec_xr32_kernel(float2* __restrict__ xh, float2* __restrict__ xl, float2* __restrict__ r,
                                const float2* __restrict__ p, const float2* __restrict__ w,
                                const double2* __restrict__ alpha, const int* __restrict__ active,
                                int64_t N, double2* __restrict__ part) {
    const int e = blockIdx.y;
    if (!active[e]) return;
    __shared__ double2 red[32];
    const double2 a = alpha[e];
    float axh, axl, ayh, ayl;
    df_split(a.x, axh, axl);
    df_split(a.y, ayh, ayl);
    const int64_t o = (int64_t)e * N;
    float acc = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 pv = p[o + i], wv = w[o + i];
        float2 hv = xh[o + i], lv = xl[o + i], rv = r[o + i];
        float ph, pl;
        df_mul(axh, axl, pv.x, ph, pl); df_add(hv.x, lv.x, ph, pl);      // re += ax px - ay py
        df_mul(ayh, ayl, pv.y, ph, pl); df_add(hv.x, lv.x, -ph, -pl);
        df_mul(axh, axl, pv.y, ph, pl); df_add(hv.y, lv.y, ph, pl);      // im += ax py + ay px
        df_mul(ayh, ayl, pv.x, ph, pl); df_add(hv.y, lv.y, ph, pl);
        rv.x -= axh * wv.x - ayh * wv.y;
        rv.y -= axh * wv.y + ayh * wv.x;
        xh[o + i] = hv;
        xl[o + i] = lv;
        r[o + i] = rv;
        acc += rv.x * rv.x + rv.y * rv.y;
    }
    const double2 t = block_sum2(make_double2((double)acc, 0.0), red);
    if (threadIdx.x == 0) part[(int64_t)e * gridDim.x + blockIdx.x] = t;
}

// p = z + beta p (beta = 0 with copy = 1: p = z), FP32
__global__ void vec_p32_kernel(float2* __restrict__ p, const float2* __restrict__ z,
                               const double2* __restrict__ beta, const int* __restrict__ active,
                               int64_t N, int copy) {
    const int e = blockIdx.y;
    if (!active[e]) return;
    const float2 b = copy ? make_float2(0.f, 0.f) : make_float2((float)beta[e].x, (float)beta[e].y);
    const int64_t o = (int64_t)e * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 zv = z[o + i];
        const float2 pv = copy ? make_float2(0.f, 0.f) : p[o + i];
        p[o + i] = make_float2(zv.x + b.x * pv.x - b.y * pv.y, zv.y + b.x * pv.y + b.y * pv.x);
    }
}

// x += xh + xl, increment = 0, for the energies with mask set (all if null)
__global__ void vec_fold_kernel(double2* __restrict__ x, float2* __restrict__ xh, float2* __restrict__ xl,
                                const int* __restrict__ mask, int64_t N) {
    const int e = blockIdx.y;
    if (mask && !mask[e]) return;
    const int64_t o = (int64_t)e * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 hv = xh[o + i], lv = xl[o + i];
        double2 xv = x[o + i];
        xv.x += (double)hv.x + (double)lv.x;
        xv.y += (double)hv.y + (double)lv.y;
        x[o + i] = xv;
        xh[o + i] = make_float2(0.f, 0.f);
        xl[o + i] = make_float2(0.f, 0.f);
    }
}

// r = f - t (FP64, t = A x), stored rounded to complex64, for the energies
// with upd set; partial ||f - t||^2 in FP64
__global__ void vec_res32_kernel(const double2* __restrict__ f, const double2* __restrict__ t,
                                 float2* __restrict__ r, const int* __restrict__ upd, int64_t N,
                                 double2* __restrict__ part) {
    const int e = blockIdx.y;
    if (!upd[e]) return;
    __shared__ double2 red[32];
    const int64_t o = (int64_t)e * N;
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 fv = f[i], tv = t[o + i];
        const double2 rv = make_double2(fv.x - tv.x, fv.y - tv.y);
        r[o + i] = make_float2((float)rv.x, (float)rv.y);
        acc.x += rv.x * rv.x + rv.y * rv.y;
    }
    const double2 s = block_sum2(acc, red);
    if (threadIdx.x == 0) part[(int64_t)e * gridDim.x + blockIdx.x] = s;
}

int vec_init32(const void* f, void* x, void* r, void* xh, void* xl, int64_t N, int nE, cudaStream_t st) {
    vec_init32_kernel<<<1024, 256, 0, st>>>((const double2*)f, (double2*)x, (float2*)r, (float2*)xh,
                                            (float2*)xl, N, nE);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}
int vec_xr32(void* xh, void* xl, void* r, const void* p, const void* w, const double2* alpha, const int* act,
             int64_t N, int nE, double2* part, int nparts, cudaStream_t st) {
    vec_xr32_kernel<<<dim3(nparts, nE), 256, 0, st>>>((float2*)xh, (float2*)xl, (float2*)r, (const float2*)p,
                                                       (const float2*)w, alpha, act, N, part);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}
int vec_p32(void* p, const void* z, const double2* beta, const int* act, int64_t N, int nE, int copy,
            cudaStream_t st) {
    vec_p32_kernel<<<dim3(256, nE), 256, 0, st>>>((float2*)p, (const float2*)z, beta, act, N, copy);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}
int vec_fold(void* x, void* xh, void* xl, const int* mask, int64_t N, int nE, cudaStream_t st) {
    vec_fold_kernel<<<dim3(256, nE), 256, 0, st>>>((double2*)x, (float2*)xh, (float2*)xl, mask, N);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}
int vec_res32(const void* f, const void* t, void* r, const int* upd, int64_t N, int nE, double2* part,
              int nparts, cudaStream_t st) {
    vec_res32_kernel<<<dim3(nparts, nE), 256, 0, st>>>((const double2*)f, (const double2*)t, (float2*)r, upd,
                                                        N, part);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

// ------------------------------------------------- flexible GCR (truncated)
// c_j = <Q_j, q> (Hermitian) for the mu stored directions j != slot
__global__ void gcr_dots_kernel(const double2* __restrict__ Q, int64_t slot_stride, int mu, int ld, int slot,
                                const int* __restrict__ active, int64_t N, double2* __restrict__ part) {
    const int e = blockIdx.y;
    if (!active[e]) return;
    __shared__ double2 red[32];
    const int64_t o = (int64_t)e * N;
    const double2* q = Q + slot * slot_stride + o;
    for (int j = 0; j < mu; ++j) {
        double2 acc = make_double2(0.0, 0.0);
        if (j != slot) {
            const double2* qj = Q + j * slot_stride + o;
            for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
                 i += (int64_t)gridDim.x * blockDim.x) {
                const double2 a = qj[i], b = q[i];
                acc.x += a.x * b.x + a.y * b.y;        // conj(a) b
                acc.y += a.x * b.y - a.y * b.x;
            }
        }
        const double2 t = block_sum2(acc, red);
        if (threadIdx.x == 0) part[((int64_t)e * ld + j) * gridDim.x + blockIdx.x] = t;
    }
}

// beta_j = c_j / <Q_j, Q_j> per energy (one thread per (energy, j))
__global__ void gcr_beta_kernel(const double2* __restrict__ part, int nparts, int mu, int ld, int slot,
                                const double* __restrict__ qnorm, const int* __restrict__ active,
                                int nE, double2* __restrict__ beta) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    const int e = id / mu, j = id % mu;
    if (e >= nE || !active[e]) return;
    double2 t = make_double2(0.0, 0.0);
    if (j != slot) {
        for (int i = 0; i < nparts; ++i) { t.x += part[((int64_t)e * ld + j) * nparts + i].x; t.y += part[((int64_t)e * ld + j) * nparts + i].y; }
        const double qn = qnorm[(int64_t)e * ld + j];
        t.x /= qn; t.y /= qn;
    }
    beta[(int64_t)e * ld + j] = t;
}

// P_s -= sum_j beta_j P_j, Q_s -= sum_j beta_j Q_j; partials of <Q_s,Q_s> and <Q_s, r>
__global__ void gcr_update_kernel(double2* __restrict__ Pb, double2* __restrict__ Q, int64_t slot_stride,
                                  int mu, int ld, int slot, const double2* __restrict__ beta,
                                  const double2* __restrict__ r, const int* __restrict__ active,
                                  int64_t N, double2* __restrict__ p1, double2* __restrict__ p2) {
    const int e = blockIdx.y;
    if (!active[e]) return;
    __shared__ double2 red[32];
    const int64_t o = (int64_t)e * N;
    double2 a1 = make_double2(0.0, 0.0), a2 = make_double2(0.0, 0.0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double2 pv = Pb[slot * slot_stride + o + i], qv = Q[slot * slot_stride + o + i];
        for (int j = 0; j < mu; ++j) {
            if (j == slot) continue;
            const double2 b = beta[(int64_t)e * ld + j];
            const double2 pj = Pb[j * slot_stride + o + i], qj = Q[j * slot_stride + o + i];
            pv.x -= b.x * pj.x - b.y * pj.y; pv.y -= b.x * pj.y + b.y * pj.x;
            qv.x -= b.x * qj.x - b.y * qj.y; qv.y -= b.x * qj.y + b.y * qj.x;
        }
        Pb[slot * slot_stride + o + i] = pv;
        Q[slot * slot_stride + o + i] = qv;
        const double2 rv = r[o + i];
        a1.x += qv.x * qv.x + qv.y * qv.y;
        a2.x += qv.x * rv.x + qv.y * rv.y;          // conj(q) r
        a2.y += qv.x * rv.y - qv.y * rv.x;
    }
    const double2 t1 = block_sum2(a1, red);
    if (threadIdx.x == 0) p1[(int64_t)e * gridDim.x + blockIdx.x] = t1;
    const double2 t2 = block_sum2(a2, red);
    if (threadIdx.x == 0) p2[(int64_t)e * gridDim.x + blockIdx.x] = t2;
}

// nq_s = <Q_s, Q_s>, alpha = <Q_s, r>/nq_s
__global__ void gcr_alpha_kernel(const double2* __restrict__ p1, const double2* __restrict__ p2, int nparts,
                                 int ld, int slot, double* __restrict__ qnorm, PcgState s, int nE) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nE || !s.active[e]) return;
    double n = 0;
    double2 c = make_double2(0.0, 0.0);
    for (int i = 0; i < nparts; ++i) {
        n += p1[(int64_t)e * nparts + i].x;
        c.x += p2[(int64_t)e * nparts + i].x;
        c.y += p2[(int64_t)e * nparts + i].y;
    }
    if (!(n > 0.0) || !isfinite(n)) {
        retire(s, e, SOFT_ERR_BREAKDOWN);
        return;
    }
    qnorm[(int64_t)e * ld + slot] = n;
    s.alpha[e] = make_double2(c.x / n, c.y / n);
}

int gcr_step(int phase, void* Pb, void* Q, int64_t slot_stride, int mu, int ld, int slot, double2* beta,
             double* qnorm, const void* r, const int* act, int64_t N, int nE, double2* gpart, double2* part,
             double2* part2, int nparts, const PcgState& s, cudaStream_t st) {
    if (phase == 0) {
        if (mu > 1) {
            gcr_dots_kernel<<<dim3(nparts, nE), 256, 0, st>>>((const double2*)Q, slot_stride, mu, ld, slot, act, N, gpart);
            gcr_beta_kernel<<<(nE * mu + 127) / 128, 128, 0, st>>>(gpart, nparts, mu, ld, slot, qnorm, act, nE, beta);
        }
        gcr_update_kernel<<<dim3(nparts, nE), 256, 0, st>>>((double2*)Pb, (double2*)Q, slot_stride, mu, ld, slot,
                                                            beta, (const double2*)r, act, N, part, part2);
        gcr_alpha_kernel<<<(nE + 63) / 64, 64, 0, st>>>(part, part2, nparts, ld, slot, qnorm, s, nE);
    }
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

int pcg_scalars(int stage, int nE, const double2* part, int nparts, const PcgState& s,
                cudaStream_t st, const double2* part2) {
    pcg_scalar_kernel<<<stage == STAGE_FNORM ? 1 : nE, 32, 0, st>>>(stage, nE, part, nparts, s, part2);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

}  // namespace soft
