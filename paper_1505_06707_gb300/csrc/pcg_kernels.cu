// Complex-symmetric CG (Sec. III) for the 2D stationary ECS equation:
// instantiations of the A-apply and preconditioner passes (complex128) and the
// vector / scalar kernels of the iteration.
#include "pcg.cuh"
#include "pcg_launch.h"

namespace soft {

namespace {

constexpr int TWP = 2;    // columns per CTA in the column passes (complex128)

template <int LN, int LE, int LR>
int row_kernels(int which, const PcgGeo& g, const void* a, void* b, const void* c, const double* E,
                const int* act, double2* part, int nE, cudaStream_t st) {
    using K = Cfg1D<double, LN, LE, LR>;
    const size_t smem = sizeof(double2) * 2 * K::N + 64;
    dim3 grid(g.ny, nE);
    if (which == 0) {
        auto k = a_row_kernel<double, LN, LE, LR>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return SOFT_ERR_CUDA;
        if (nE > 0) k<<<grid, K::T, smem, st>>>(g, a, b, E, act);
    } else if (which == 1) {
        auto k = pc_row1_kernel<double, LN, LE, LR>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return SOFT_ERR_CUDA;
        if (nE > 0) k<<<grid, K::T, smem, st>>>(g, a, b, act);
    } else {
        auto k = pc_row2_kernel<double, LN, LE, LR>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return SOFT_ERR_CUDA;
        if (nE > 0) k<<<grid, K::T, smem, st>>>(g, a, b, c, act, part);
    }
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

template <int LN, int LE, int LR>
int col_kernels(int which, const PcgGeo& g, const void* a, void* b, const double* E,
                const int* act, double2* part, int nE, cudaStream_t st) {
    using K = Cfg1D<double, LN, LE, LR>;
    const size_t smem = sizeof(double2) * 2 * TWP * K::N + 64;
    dim3 grid(g.nx / TWP, nE);
    if (which == 0) {
        auto k = a_col_kernel<double, LN, LE, LR, TWP>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return SOFT_ERR_CUDA;
        if (nE > 0) k<<<grid, TWP * K::T, smem, st>>>(g, a, b, act, part, (int)grid.x);
    } else {
        auto k = pc_col_kernel<double, LN, LE, LR, TWP>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return SOFT_ERR_CUDA;
        if (nE > 0) k<<<grid, TWP * K::T, smem, st>>>(g, b, E, act);
    }
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

// preconditioner passes computing in FP32 (complex128 r in, complex128 z out)
constexpr int TWP32 = 4;  // columns per CTA of the FP32 column pass

template <int LN, int LE, int LR>
int pc32_row(int which, const PcgGeo& g, const void* a, void* b, const void* c, const int* act,
             double2* part, int nE, cudaStream_t st) {
    using K = Cfg1D<float, LN, LE, LR>;
    const size_t smem = sizeof(float2) * 2 * K::N + 64;
    dim3 grid(g.ny, nE);
    if (which == 1) {
        auto k = pc_row1_kernel<float, LN, LE, LR>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return SOFT_ERR_CUDA;
        if (nE > 0) k<<<grid, K::T, smem, st>>>(g, a, b, act);
    } else {
        auto k = pc_row2_kernel<float, LN, LE, LR>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return SOFT_ERR_CUDA;
        if (nE > 0) k<<<grid, K::T, smem, st>>>(g, a, b, c, act, part);
    }
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

template <int LN, int LE, int LR>
int pc32_col(const PcgGeo& g, void* b, const double* E, const int* act, int nE, cudaStream_t st) {
    using K = Cfg1D<float, LN, LE, LR>;
    const size_t smem = sizeof(float2) * 2 * TWP32 * K::N + 64;
    dim3 grid(g.nx / TWP32, nE);
    auto k = pc_col_kernel<float, LN, LE, LR, TWP32>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return SOFT_ERR_CUDA;
    if (nE > 0) k<<<grid, TWP32 * K::T, smem, st>>>(g, b, E, act);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

// A computing in FP32
constexpr int TWA32 = 4;  // columns per CTA of the FP32 A column pass

template <int LN, int LE, int LR>
int a32_row(const PcgGeo& g, const void* a, void* b, const double* E, const int* act, int nE,
            cudaStream_t st) {
    using K = Cfg1D<float, LN, LE, LR>;
    const size_t smem = sizeof(float2) * 2 * K::N + 64;
    auto k = a_row_kernel<float, LN, LE, LR>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return SOFT_ERR_CUDA;
    if (nE > 0) k<<<dim3(g.ny, nE), K::T, smem, st>>>(g, a, b, E, act);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

template <int LN, int LE, int LR>
int a32_col(const PcgGeo& g, const void* a, void* b, const int* act, double2* part, int pstride, int nE,
            cudaStream_t st) {
    using K = Cfg1D<float, LN, LE, LR>;
    const size_t smem = sizeof(float2) * 2 * TWA32 * K::N + 64;
    auto k = a_col_kernel<float, LN, LE, LR, TWA32>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return SOFT_ERR_CUDA;
    const int nb = g.nx / TWA32;
    if (nE > 0) k<<<dim3(nb, nE), TWA32 * K::T, smem, st>>>(g, a, b, act, part, pstride > nb ? pstride : nb);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

}  // namespace

int pcg_a32_row(int logn, const PcgGeo& g, const void* p, void* w, const double* E, const int* act,
                int nE, cudaStream_t st) {
    switch (logn) {
    case 8: return a32_row<8, 3, 3>(g, p, w, E, act, nE, st);
    case 9: return a32_row<9, 3, 3>(g, p, w, E, act, nE, st);
    case 10: return a32_row<10, 3, 3>(g, p, w, E, act, nE, st);
    case 11: return a32_row<11, 3, 3>(g, p, w, E, act, nE, st);
    }
    return SOFT_ERR_UNSUPPORTED;
}

int pcg_a32_col(int logn, const PcgGeo& g, const void* p, void* w, const int* act, double2* part,
                int pstride, int nE, cudaStream_t st) {
    switch (logn) {
    case 8: return a32_col<8, 3, 3>(g, p, w, act, part, pstride, nE, st);
    case 9: return a32_col<9, 3, 3>(g, p, w, act, part, pstride, nE, st);
    case 10: return a32_col<10, 3, 3>(g, p, w, act, part, pstride, nE, st);
    case 11: return a32_col<11, 3, 3>(g, p, w, act, part, pstride, nE, st);
    }
    return SOFT_ERR_UNSUPPORTED;
}

int pcg_a32_col_blocks(int nx) { return nx / TWA32; }

int pcg_pc32_row(int logn, int which, const PcgGeo& g, const void* a, void* b, const void* c,
                 const int* act, double2* part, int nE, cudaStream_t st) {
    switch (logn) {
    case 8: return pc32_row<8, 3, 3>(which, g, a, b, c, act, part, nE, st);
    case 9: return pc32_row<9, 3, 3>(which, g, a, b, c, act, part, nE, st);
    case 10: return pc32_row<10, 3, 3>(which, g, a, b, c, act, part, nE, st);
    case 11: return pc32_row<11, 3, 3>(which, g, a, b, c, act, part, nE, st);
    }
    return SOFT_ERR_UNSUPPORTED;
}

int pcg_pc32_col(int logn, const PcgGeo& g, void* b, const double* E, const int* act, int nE,
                 cudaStream_t st) {
    switch (logn) {
    case 8: return pc32_col<8, 3, 3>(g, b, E, act, nE, st);
    case 9: return pc32_col<9, 3, 3>(g, b, E, act, nE, st);
    case 10: return pc32_col<10, 3, 3>(g, b, E, act, nE, st);
    case 11: return pc32_col<11, 3, 3>(g, b, E, act, nE, st);
    }
    return SOFT_ERR_UNSUPPORTED;
}

int pcg_row(int logn, int which, const PcgGeo& g, const void* a, void* b, const void* c,
            const double* E, const int* act, double2* part, int nE, cudaStream_t st) {
    switch (logn) {
    case 8: return row_kernels<8, 3, 3>(which, g, a, b, c, E, act, part, nE, st);
    case 9: return row_kernels<9, 3, 3>(which, g, a, b, c, E, act, part, nE, st);
    case 10: return row_kernels<10, 3, 3>(which, g, a, b, c, E, act, part, nE, st);
    case 11: return row_kernels<11, 3, 3>(which, g, a, b, c, E, act, part, nE, st);
    }
    return SOFT_ERR_UNSUPPORTED;
}

int pcg_col(int logn, int which, const PcgGeo& g, const void* a, void* b, const double* E,
            const int* act, double2* part, int nE, cudaStream_t st) {
    switch (logn) {
    case 8: return col_kernels<8, 3, 3>(which, g, a, b, E, act, part, nE, st);
    case 9: return col_kernels<9, 3, 3>(which, g, a, b, E, act, part, nE, st);
    case 10: return col_kernels<10, 3, 3>(which, g, a, b, E, act, part, nE, st);
    case 11: return col_kernels<11, 3, 3>(which, g, a, b, E, act, part, nE, st);
    }
    return SOFT_ERR_UNSUPPORTED;
}

int pcg_col_blocks(int nx) { return nx / TWP; }

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

// r = f - t (t = A x in FP64) for the energies with upd set; partial ||r||^2
__global__ void vec_res_kernel(const double2* __restrict__ f, const double2* __restrict__ t,
                               double2* __restrict__ r, const int* __restrict__ upd, int64_t N,
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
        r[o + i] = rv;
        acc.x += rv.x * rv.x + rv.y * rv.y;
    }
    const double2 s = block_sum2(acc, red);
    if (threadIdx.x == 0) part[(int64_t)e * gridDim.x + blockIdx.x] = s;
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

// per-energy scalar updates of the iteration (one thread per energy; the
// partial sums are added in a fixed order, so results are reproducible)
__global__ void pcg_scalar_kernel(int stage, int nE, const double2* __restrict__ part, int nparts,
                                  PcgState s, const double2* __restrict__ part2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (stage == STAGE_FNORM) {
        if (e == 0) {
            double t = 0;
            for (int i = 0; i < nparts; ++i) t += part[i].x;
            *s.fnorm2 = t;
        }
        return;
    }
    if (e >= nE || !s.active[e]) return;
    if (stage == STAGE_TRUE && !s.upd[e]) return;
    double2 t = make_double2(0.0, 0.0);
    for (int i = 0; i < nparts; ++i) { t.x += part[(int64_t)e * nparts + i].x; t.y += part[(int64_t)e * nparts + i].y; }
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
        if (!(rel < 0.5 * s.rref[e]) && !(s.mode[e] & 1)) {
            s.mode[e] = 3;
            s.act32[e] = 0;
            s.act64[e] = 1;
        }
        s.rref[e] = rel;
    } else if (stage == STAGE_BETA_FLEX) {
        // flexible (Polak-Ribiere) beta = z'^T (r' - r) / rho = -alpha z'^T w / rho
        double2 u = make_double2(0.0, 0.0);
        for (int i = 0; i < nparts; ++i) { u.x += part2[(int64_t)e * nparts + i].x; u.y += part2[(int64_t)e * nparts + i].y; }
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
int vec_res(const void* f, const void* t, void* r, const int* upd, int64_t N, int nE, double2* part,
            int nparts, cudaStream_t st) {
    vec_res_kernel<<<dim3(nparts, nE), 256, 0, st>>>((const double2*)f, (const double2*)t, (double2*)r, upd,
                                                      N, part);
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
    pcg_scalar_kernel<<<(nE + 63) / 64, 64, 0, st>>>(stage, nE, part, nparts, s, part2);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

}  // namespace soft
