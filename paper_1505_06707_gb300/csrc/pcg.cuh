// Stationary ECS equation A psi = f (Sec. III, Eq. linsys) on a 2D grid:
//   A = F^-1 (Kx + Ky) F + C_x (x) I + I (x) C_y + U - E.
// Because K is a sum, F^-1 Kx F = F_x^-1 Kx F_x acts along rows only and
// F^-1 Ky F = F_y^-1 Ky F_y along columns only, so A p is one row pass
// (x kinetic + C_x + U - E) plus one column pass (y kinetic + C_y) over p.
//
// The preconditioner P^-1 = F^-1 X^T (Lambda - E)^-1 X F (Eq. PreconFFT_ECS;
// Eq. PreconFFT is the same with one-wide bands and lambda = k^2/2) is
// separable, X = X_x (x) X_y, Lambda = lambda_x + lambda_y:
//   row pass 1: F_x then the band rows of X_x         (natural nu order)
//   column pass: F_y, X_y, / (lambda_x + lambda_y - E), X_y^T, F_y^-1
//   row pass 2: X_x^T then F_x^-1
// The paper's F has e^{+i k x}: conj(FFT(conj(.))) gives that sum with the
// forward FFT; the x_0 phase and 1/sqrt N are folded into the band tables.
//
// Batched over energies: grid.y (or grid.z) = energy; converged energies are
// masked out by the active flags.
#pragma once
#include "soft1d.cuh"

namespace soft {

struct PcgGeo {
    int nx, ny;
    const void* Wx; const void* Wy;        // pass twiddles
    const void* Kx; const void* Ky;        // k^2/(2n) in each FFT's output order (phase-table format)
    const void* U;                          // U(z(x), z(y)) [ny][nx], complex
    const void* Cx; const void* Cy;        // C tridiagonals, 3*n complex (sub, diag, sup)
    int nbx, blk0x, nby, blk0y;            // strip blocks
    // preconditioner tables per axis (natural index order)
    const int* posx; const int* posy;      // FFT output position of natural index
    const int* bsx; const int* bsy;        // band start
    const int* bwx; const int* bwy;        // band width
    // band rows, u-major: entry u of row nu at [u * n + nu], zero past the
    // row's width, so that one u of consecutive rows is one contiguous load
    const void* xfx; const void* xfy;      // forward band rows (complex)
    const void* xbx; const void* xby;      // backward band rows (complex)
    const void* lamx; const void* lamy;    // eigenvalues (complex)
    int64_t N;                              // nx * ny
};

template <typename C>
__device__ __forceinline__ C cconj(C a) { return cmk<C>(a.x, -a.y); }

// complex value in another precision
template <typename C, typename D>
__device__ __forceinline__ C cto(D a) { return cmk<C>((decltype(C::x))a.x, (decltype(C::x))a.y); }

// block reduction of a complex FP64 value; returns the total in thread 0
__device__ __forceinline__ double2 block_sum2(double2 v, double2* red) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double2 t = make_double2(0.0, 0.0);
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) { t.x += red[i].x; t.y += red[i].y; }
    return t;
}

// shared-memory pitch of one column in the column passes: N + 64 bytes, so
// that the TW columns of one row fall in different banks when the tile is
// filled and drained row by row
template <typename C, int N>
struct ColPitch { static constexpr int value = N + 64 / (int)sizeof(C); };

// --------------------------------------------------------------- A apply
// w = F_x^-1 Kx F_x p + C_x p + (U - E) p, one CTA per (row, energy); p and w
// are IO (complex128 or complex64), the pass computes in R (with R = float
// the tables are FP32)
template <typename R, typename IO, int LOGN, int LOGE, int LOGRM>
__global__ void __launch_bounds__(Cfg1D<R, LOGN, LOGE, LOGRM>::T, Cfg1D<R, LOGN, LOGE, LOGRM>::MINB)
a_row_kernel(PcgGeo g, const void* __restrict__ p_v, void* __restrict__ w_v,
             const double* __restrict__ E, const int* __restrict__ active)
{
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    using TT = typename K::TT;
    constexpr int N = K::N, T = K::T, E_ = K::E;
    const int y = blockIdx.x, e = blockIdx.y;
    if (active && !active[e]) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* S = reinterpret_cast<C*>(smem_raw);
    C* P0 = S + N;                               // p row kept for C_x p and (U - E) p
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)e * g.N + (int64_t)y * N;
    const IO* __restrict__ p = reinterpret_cast<const IO*>(p_v) + base;
    IO* __restrict__ w = reinterpret_cast<IO*>(w_v) + base;
    const C* W = reinterpret_cast<const C*>(g.Wx);
    for (int j = 0; j < E_; ++j) {
        const int n = tid + j * T;
        const C v = cto<C>(p[n]);
        S[swz<C>(n)] = v;
        P0[n] = v;
    }
    __syncthreads();
    fwd_fft<R, LOGN, LOGE, LOGRM, 0>(S, W, tid);
    kmul<R, LOGN, LOGE, LOGRM>(S, reinterpret_cast<const TT*>(g.Kx), tid);
    inv_fft<R, LOGN, LOGE, LOGRM, K::NPASS - 1>(S, W, tid);
    const C* __restrict__ U = reinterpret_cast<const C*>(g.U) + (int64_t)y * N;
    const C* __restrict__ Cx = reinterpret_cast<const C*>(g.Cx);
    const R En = (R)E[e];
    for (int j = 0; j < E_; ++j) {
        const int n = tid + j * T;
        const C pv = P0[n];
        C u = __ldg(&U[n]);
        u.x -= En;
        C v = cfma(u, pv, S[swz<C>(n)]);
        if (((n - g.blk0x) & (N - 1)) < g.nbx) {
            v = cfma(__ldg(&Cx[n]), P0[(n + N - 1) & (N - 1)], v);
            v = cfma(__ldg(&Cx[N + n]), pv, v);
            v = cfma(__ldg(&Cx[2 * N + n]), P0[(n + 1) & (N - 1)], v);
        }
        w[n] = cto<IO>(v);
    }
}

// w += F_y^-1 Ky F_y p + C_y p, TW columns per CTA; partial of p^T w per CTA
// at part[e * pstride + block], the entries from gridDim.x to pstride zeroed
// (p and w IO, the pass computes in R; each thread sums its terms of p^T w
// in IO precision, the block sum is FP64)
template <typename R, typename IO, int LOGN, int LOGE, int LOGRM, int TW, int MINB = 1>
__global__ void __launch_bounds__(TW * Cfg1D<R, LOGN, LOGE, LOGRM>::T, MINB)
a_col_kernel(PcgGeo g, const void* __restrict__ p_v, void* __restrict__ w_v,
             const int* __restrict__ active, double2* __restrict__ part, int pstride)
{
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    using TT = typename K::TT;
    constexpr int N = K::N, T = K::T, NIT = N / T, PITCH = ColPitch<C, N>::value;
    const int e = blockIdx.y;
    if (active && !active[e]) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* S = reinterpret_cast<C*>(smem_raw);
    C* P0 = S + TW * PITCH;
    __shared__ double2 red[32];
    const int c0 = blockIdx.x * TW, nx = g.nx;
    const int64_t eb = (int64_t)e * g.N;
    const IO* __restrict__ p = reinterpret_cast<const IO*>(p_v) + eb;
    IO* __restrict__ w = reinterpret_cast<IO*>(w_v) + eb;
#pragma unroll
    for (int it = 0; it < NIT; ++it) {              // row by row: the TW columns of a row are adjacent
        const int idx = threadIdx.x + it * TW * T;
        const int yy = idx / TW, j = idx % TW;
        const C v = cto<C>(p[(int64_t)yy * nx + c0 + j]);
        S[j * PITCH + swz<C>(yy)] = v;
        P0[j * PITCH + yy] = v;
    }
    __syncthreads();
    const int col = threadIdx.x / T, tid = threadIdx.x % T;
    C* Sc = S + col * PITCH;
    const C* W = reinterpret_cast<const C*>(g.Wy);
    fwd_fft<R, LOGN, LOGE, LOGRM, 0>(Sc, W, tid);
    kmul<R, LOGN, LOGE, LOGRM>(Sc, reinterpret_cast<const TT*>(g.Ky), tid);
    inv_fft<R, LOGN, LOGE, LOGRM, K::NPASS - 1>(Sc, W, tid);
    const C* __restrict__ Cy = reinterpret_cast<const C*>(g.Cy);
    IO acc = cmk<IO>(0, 0);
#pragma unroll 4
    for (int it = 0; it < NIT; ++it) {
        const int idx = threadIdx.x + it * TW * T;
        const int yy = idx / TW, j = idx % TW;
        const C* Pj = P0 + j * PITCH;
        C v = S[j * PITCH + swz<C>(yy)];
        if (((yy - g.blk0y) & (N - 1)) < g.nby) {
            v = cfma(__ldg(&Cy[yy]), Pj[(yy + N - 1) & (N - 1)], v);
            v = cfma(__ldg(&Cy[N + yy]), Pj[yy], v);
            v = cfma(__ldg(&Cy[2 * N + yy]), Pj[(yy + 1) & (N - 1)], v);
        }
        const int64_t a = (int64_t)yy * nx + c0 + j;
        const IO wv = cto<IO>(cadd(cto<C>(w[a]), v));
        w[a] = wv;
        const IO pv = cto<IO>(Pj[yy]);
        acc.x += pv.x * wv.x - pv.y * wv.y;      // bilinear p^T w
        acc.y += pv.x * wv.y + pv.y * wv.x;
    }
    const double2 t = block_sum2(cto<double2>(acc), red);
    if (threadIdx.x == 0) {
        part[(int64_t)e * pstride + blockIdx.x] = t;
        for (int k = blockIdx.x + gridDim.x; k < pstride; k += gridDim.x)
            part[(int64_t)e * pstride + k] = make_double2(0.0, 0.0);
    }
}

// --------------------------------------------------------- preconditioner
// band mat-vec for NJ rows nu_j = nu0 + j step at once (independent chains):
// out[j] = sum_{u < width} tab[u * n + nu_j] * in(start[nu_j] + u).  The
// tables are zero past each row's width, so every row runs to the widest of
// the NJ with its input index clamped to n - 1.
template <typename C, int NJ, class In>
__device__ __forceinline__ void band_rows(int nu0, int step, int n, const int* __restrict__ bs,
                                          const int* __restrict__ bw, const C* __restrict__ tab, In in,
                                          C (&out)[NJ]) {
    int s0[NJ], wm = 0;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        s0[j] = __ldg(&bs[nu0 + j * step]);
        wm = max(wm, __ldg(&bw[nu0 + j * step]));
        out[j].x = 0; out[j].y = 0;
    }
    for (int u = 0; u < wm; ++u) {
#pragma unroll
        for (int j = 0; j < NJ; ++j)
            out[j] = cfma(__ldg(&tab[u * n + nu0 + j * step]), in(min(s0[j] + u, n - 1)), out[j]);
    }
}
constexpr int BAND_NJ = 4;     // band rows per thread at once

// row pass 1: t = X_x F_x r (F with e^{+ikx}), natural nu order
// (r is IO; the pass computes in R: t and the tables are in R)
template <typename R, typename IO, int LOGN, int LOGE, int LOGRM>
__global__ void __launch_bounds__(Cfg1D<R, LOGN, LOGE, LOGRM>::T, Cfg1D<R, LOGN, LOGE, LOGRM>::MINB)
pc_row1_kernel(PcgGeo g, const void* __restrict__ r_v, void* __restrict__ t_v,
               const int* __restrict__ active)
{
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    constexpr int N = K::N, T = K::T, E_ = K::E;
    static_assert(E_ % BAND_NJ == 0, "band rows per thread");
    const int y = blockIdx.x, e = blockIdx.y;
    if (active && !active[e]) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* S = reinterpret_cast<C*>(smem_raw);
    C* Fn = S + N;                               // F_x r in natural index order
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)e * g.N + (int64_t)y * N;
    const IO* __restrict__ r = reinterpret_cast<const IO*>(r_v) + base;
    C* __restrict__ t = reinterpret_cast<C*>(t_v) + base;
    for (int j = 0; j < E_; ++j) {
        const int n = tid + j * T;
        S[swz<C>(n)] = cconj(cto<C>(r[n]));
    }
    __syncthreads();
    fwd_fft<R, LOGN, LOGE, LOGRM, 0>(S, reinterpret_cast<const C*>(g.Wx), tid);
    for (int j = 0; j < E_; ++j) {
        const int m = tid + j * T;
        Fn[m] = cconj(S[swz<C>(__ldg(&g.posx[m]))]);
    }
    __syncthreads();
    const C* xf = reinterpret_cast<const C*>(g.xfx);
    for (int j0 = 0; j0 < E_; j0 += BAND_NJ) {
        C o[BAND_NJ];
        band_rows<C, BAND_NJ>(tid + j0 * T, T, N, g.bsx, g.bwx, xf, [&](int m) { return Fn[m]; }, o);
#pragma unroll
        for (int j = 0; j < BAND_NJ; ++j) t[tid + (j0 + j) * T] = o[j];
    }
}

// column pass: F_y, X_y, / (lambda_x + lambda_y - E), X_y^T, F_y^-1 (in place on t)
template <typename R, int LOGN, int LOGE, int LOGRM, int TW, int MINB = 1>
__global__ void __launch_bounds__(TW * Cfg1D<R, LOGN, LOGE, LOGRM>::T, MINB)
pc_col_kernel(PcgGeo g, void* __restrict__ t_v, const double* __restrict__ E,
              const int* __restrict__ active)
{
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    constexpr int N = K::N, T = K::T, E_ = K::E, PITCH = ColPitch<C, N>::value;
    static_assert(E_ % BAND_NJ == 0, "band rows per thread");
    const int e = blockIdx.y;
    if (active && !active[e]) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* S = reinterpret_cast<C*>(smem_raw);
    C* S2 = S + TW * PITCH;
    const int c0 = blockIdx.x * TW, nx = g.nx;
    C* __restrict__ t = reinterpret_cast<C*>(t_v) + (int64_t)e * g.N;
#pragma unroll
    for (int it = 0; it < E_; ++it) {
        const int idx = threadIdx.x + it * TW * T;
        const int yy = idx / TW, j = idx % TW;
        S[j * PITCH + swz<C>(yy)] = cconj(t[(int64_t)yy * nx + c0 + j]);
    }
    __syncthreads();
    const int col = threadIdx.x / T, tid = threadIdx.x % T;
    C* Sc = S + col * PITCH;
    C* S2c = S2 + col * PITCH;
    const C* W = reinterpret_cast<const C*>(g.Wy);
    fwd_fft<R, LOGN, LOGE, LOGRM, 0>(Sc, W, tid);
    for (int j = 0; j < E_; ++j) {                 // F_y t in natural index order
        const int m = tid + j * T;
        S2c[m] = cconj(Sc[swz<C>(__ldg(&g.posy[m]))]);
    }
    __syncthreads();
    const int nu = c0 + col;
    const C lx = reinterpret_cast<const C*>(g.lamx)[nu];
    const R En = (R)E[e];
    const C* xf = reinterpret_cast<const C*>(g.xfy);
    const C* xb = reinterpret_cast<const C*>(g.xby);
    const C* ly = reinterpret_cast<const C*>(g.lamy);
    for (int j0 = 0; j0 < E_; j0 += BAND_NJ) {    // X_y, then the eigenvalue denominator
        C o[BAND_NJ];
        band_rows<C, BAND_NJ>(tid + j0 * T, T, N, g.bsy, g.bwy, xf, [&](int m) { return S2c[m]; }, o);
#pragma unroll
        for (int j = 0; j < BAND_NJ; ++j) {
            const int mu = tid + (j0 + j) * T;
            const C lm = __ldg(&ly[mu]);
            const C den = cmk<C>(lx.x + lm.x - En, lx.y + lm.y);
            const R dn = den.x * den.x + den.y * den.y;
            Sc[mu] = cscale(cmulc(o[j], den), (R)1 / dn);    // c / den, natural order
        }
    }
    __syncthreads();
    for (int j0 = 0; j0 < E_; j0 += BAND_NJ) {    // X_y^T into FFT positions (conjugated)
        C o[BAND_NJ];
        band_rows<C, BAND_NJ>(tid + j0 * T, T, N, g.bsy, g.bwy, xb, [&](int nu2) { return Sc[nu2]; }, o);
#pragma unroll
        for (int j = 0; j < BAND_NJ; ++j) S2c[swz<C>(__ldg(&g.posy[tid + (j0 + j) * T]))] = cconj(o[j]);
    }
    __syncthreads();
    inv_fft<R, LOGN, LOGE, LOGRM, K::NPASS - 1>(S2c, W, tid);
#pragma unroll
    for (int it = 0; it < E_; ++it) {
        const int idx = threadIdx.x + it * TW * T;
        const int yy = idx / TW, j = idx % TW;
        t[(int64_t)yy * nx + c0 + j] = cconj(S2[j * PITCH + swz<C>(yy)]);
    }
}

// row pass 2: z = F_x^-1 X_x^T t; with r, the partial of r^T z per CTA in
// part, and with w also that of z^T w in part2 (z, r and w are IO, the pass
// computes in R; each thread sums its terms in IO precision, the block sum
// is FP64)
template <typename R, typename IO, int LOGN, int LOGE, int LOGRM>
__global__ void __launch_bounds__(Cfg1D<R, LOGN, LOGE, LOGRM>::T, Cfg1D<R, LOGN, LOGE, LOGRM>::MINB)
pc_row2_kernel(PcgGeo g, const void* __restrict__ t_v, void* __restrict__ z_v,
               const void* __restrict__ r_v, const void* __restrict__ w_v, const int* __restrict__ active,
               double2* __restrict__ part, double2* __restrict__ part2)
{
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    constexpr int N = K::N, T = K::T, E_ = K::E;
    static_assert(E_ % BAND_NJ == 0, "band rows per thread");
    const int y = blockIdx.x, e = blockIdx.y;
    if (active && !active[e]) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* S = reinterpret_cast<C*>(smem_raw);
    C* Tn = S + N;
    __shared__ double2 red[32];
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)e * g.N + (int64_t)y * N;
    const C* __restrict__ t = reinterpret_cast<const C*>(t_v) + base;
    IO* __restrict__ z = reinterpret_cast<IO*>(z_v) + base;
    for (int j = 0; j < E_; ++j) {
        const int n = tid + j * T;
        Tn[n] = t[n];
    }
    __syncthreads();
    const C* xb = reinterpret_cast<const C*>(g.xbx);
    for (int j0 = 0; j0 < E_; j0 += BAND_NJ) {
        C o[BAND_NJ];
        band_rows<C, BAND_NJ>(tid + j0 * T, T, N, g.bsx, g.bwx, xb, [&](int nu) { return Tn[nu]; }, o);
#pragma unroll
        for (int j = 0; j < BAND_NJ; ++j) S[swz<C>(__ldg(&g.posx[tid + (j0 + j) * T]))] = cconj(o[j]);
    }
    __syncthreads();
    inv_fft<R, LOGN, LOGE, LOGRM, K::NPASS - 1>(S, reinterpret_cast<const C*>(g.Wx), tid);
    IO acc = cmk<IO>(0, 0), acc2 = cmk<IO>(0, 0);
    const IO* r = r_v ? reinterpret_cast<const IO*>(r_v) + base : nullptr;
    const IO* w = w_v ? reinterpret_cast<const IO*>(w_v) + base : nullptr;
    for (int j = 0; j < E_; ++j) {
        const int n = tid + j * T;
        const IO zv = cto<IO>(cconj(S[swz<C>(n)]));
        z[n] = zv;
        if (r) {
            const IO rv = r[n];
            acc.x += rv.x * zv.x - rv.y * zv.y;
            acc.y += rv.x * zv.y + rv.y * zv.x;
        }
        if (w) {
            const IO wv = w[n];
            acc2.x += zv.x * wv.x - zv.y * wv.y;
            acc2.y += zv.x * wv.y + zv.y * wv.x;
        }
    }
    if (part) {
        const double2 s = block_sum2(cto<double2>(acc), red);
        if (threadIdx.x == 0) part[(int64_t)e * gridDim.x + blockIdx.x] = s;
    }
    if (part2) {
        const double2 s = block_sum2(cto<double2>(acc2), red);
        if (threadIdx.x == 0) part2[(int64_t)e * gridDim.x + blockIdx.x] = s;
    }
}

}  // namespace soft
