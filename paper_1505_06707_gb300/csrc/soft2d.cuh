// Line passes of the 2D and 3D split-operator steps (Sec. II with
// K = K_x + K_y (+ K_z) and C = C_x + C_y (+ C_z) as Kronecker sums).
//
// The merged scheme in time order is ... V/2, CN, V/2, K, V/2, CN, V/2, K ...
// with V/2 = e^{-iU tau/2}, CN = CN_x CN_y (CN_z) and K = K_x K_y (K_z) the
// kinetic factors.  Factors acting on different axes commute, so in 2D the
// product of one step regroups into two passes over the grid, with the state
// kept in x space between them:
//   row pass    (x lines)  K_x, V/2, CN_x         (ROW_KVC)
//   column pass (y lines)  CN_y, V/2, K_y         (COL_CVK)
// so that K_y K_x | V/2 CN_x CN_y V/2 | K_y K_x ... is the paper's step
// sequence.  CN_y is the identity on the rows outside the y-strip block, so
// the 2D row pass applies their second V/2 itself and the column pass only
// that of the block rows (COL_CBK).  Each K_d is F_d, e^{-i k_d^2 tau/2} (or
// its half at the ends of a call), F_d^-1 with the last forward and first
// inverse FFT pass fused (kcenter).  ROW_K and COL_K apply the kinetic factor
// alone (the ends of a call).  The 3D step adds a strip CN pass along y
// (cn_lines_kernel) between the row pass and a COL_CVK pass along z, and a
// COL_K pass along y.
#pragma once
#include "soft1d.cuh"
#include "soft2d_geo.h"

namespace soft {

enum RowMode { ROW_K = 0, ROW_KVC = 1 };
enum ColMode { COL_K = 0, COL_CVK = 1, COL_CBK = 2 };

// Pass twiddles of the line passes.  Complex128 plans, which are bound by
// the FP64 pipe, store every W^{M off} for the passes with a stride of at
// most TWFULL_MAXS and W^{M off}, M = 1 .. 4, for the others (TwFull, as the
// complex128 1D step), so a butterfly forms no products of bases.
// Complex64 plans store the four bases W^{2^k off} per pass: their kernels
// are bound by instruction issue with shared memory busy, and the full
// tables' 15 loads per radix-16 butterfly measured slower than the 4 loads
// and the products.
template <typename R> struct Tw2D { using T = TwFull<typename CT<R>::C>; };
template <> struct Tw2D<float> { using T = float2; };

// Shared memory of the row pass: the row (swizzled) and the scan scratch of
// the strip CN, the row's e^{-iU tau/2}, the twiddles.
template <typename R, int LOGN, int LOGE, int LOGRM>
struct Cfg2DRow : Cfg1D<R, LOGN, LOGE, LOGRM> {
    using C = typename CT<R>::C;
    using VT = typename VabT<R>::T;
    using TWT = typename Tw2D<R>::T;
    static constexpr int N = 1 << LOGN;
    static constexpr int TWN = TwCountT<TWT, LOGN, LOGRM>::value;
    static constexpr size_t OFF_B = sizeof(C) * (N + 64);
    static constexpr size_t OFF_W = OFF_B + sizeof(VT) * N;
    static constexpr size_t SMEM2 = OFF_W + sizeof(TWT) * TWN;
    static_assert(OFF_B % 16 == 0 && OFF_W % 16 == 0, "16-byte aligned parts");
};

// Inverse pass 0 with post(n, v) applied to every output as it is stored
// (SH: twiddles in shared memory).
template <typename R, int LOGN, int LOGE, int LOGRM, bool SH, typename TW, class Post>
__device__ __forceinline__ void inv_pass0_post(typename CT<R>::C* S, const TW* __restrict__ W, int tid,
                                               Post post) {
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    using G = PassGeom<LOGN, LOGRM, 0>;
    constexpr int LOGR = G::LOGR, RR = 1 << LOGR;
    constexpr int s = G::S;
    constexpr bool FULL = TwLay<TW>::template full<LOGN, LOGRM, 0>();
#pragma unroll 1
    for (int u = 0; u < K::E / RR; ++u) {
        const int off = tid + u * K::T;
        const int sb = swz<C>(off);
        C v[RR];
        TW tb[FULL ? RR - 1 : 4];
        if constexpr (s > 1)
            load_tw<TW, TwLay<TW>::template rows<LOGN, LOGRM, 0>(), s, SH>(
                tb, W + TwLay<TW>::template toff<LOGN, LOGRM, 0>() + off);
        LoadInv<C, TW, RR, s, 0, FULL>::run(S, v, tb, sb, s > 1);
        dft_reg<C, RR, +1>(v);
#pragma unroll
        for (int m = 0; m < RR; ++m) S[sb ^ swz<C>(m * s)] = post(off + m * s, v[bitrev_c(m, LOGR)]);
    }
}

// One CTA per row (row blockIdx.x of the ny rows; 3D: ny nz).  The row,
// its potential factors and the twiddles are staged in shared memory by
// asynchronous copies issued together at the start.  ROW_KVC: F_x,
// e^{-i kx^2 tau/2} (the table tkx, 1/N folded in), F_x^-1 with V/2 applied
// as the last inverse pass stores, then CN_x on the x-strip block.  ROW_K:
// the kinetic factor alone.
template <typename R, int LOGN, int LOGE, int LOGRM, int MODE>
__global__ void __launch_bounds__(Cfg1D<R, LOGN, LOGE, LOGRM>::T, Cfg1D<R, LOGN, LOGE, LOGRM>::MINB)
row_pass_kernel(Geo2D g, void* __restrict__ psi_v, const void* __restrict__ tkx_v)
{
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using RC = Cfg2DRow<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    using TT = typename K::TT;
    using VT = typename VabT<R>::T;
    using TWT = typename RC::TWT;
    constexpr int N = K::N, T = K::T, E = K::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* S = reinterpret_cast<C*>(smem_raw);
    C* scan = S + N;
    VT* Tv = reinterpret_cast<VT*>(smem_raw + RC::OFF_B);
    TWT* Ws = reinterpret_cast<TWT*>(smem_raw + RC::OFF_W);
    const int tid = threadIdx.x;
    const int64_t y = blockIdx.x;
    C* __restrict__ row = reinterpret_cast<C*>(psi_v) + y * N;
    const TWT* __restrict__ W = reinterpret_cast<const TWT*>(g.Wx);
    const VT* __restrict__ tv = reinterpret_cast<const VT*>(g.TVh) + y * N;
    const TT* __restrict__ tkx = reinterpret_cast<const TT*>(tkx_v);

#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int n = tid + j * T;
        cp_async<sizeof(C)>(&S[swz<C>(n)], &row[n]);
        if constexpr (MODE == ROW_KVC) cp_async<sizeof(VT)>(&Tv[n], &tv[n]);
    }
    for (int i = tid; i < RC::TWN; i += T) cp_async<sizeof(TWT)>(&Ws[i], &W[i]);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    fwd_passes<R, LOGN, LOGE, LOGRM, 0, K::NPASS - 1>(S, Ws, tid);
    kcenter<R, LOGN, LOGE, LOGRM>(S, tkx, tid);
    __syncthreads();
    if constexpr (MODE == ROW_K) {
        inv_passes<R, LOGN, LOGE, LOGRM, K::NPASS - 2, 0>(S, Ws, tid);
    } else {
        inv_passes<R, LOGN, LOGE, LOGRM, K::NPASS - 2, 1>(S, Ws, tid);
        inv_pass0_post<R, LOGN, LOGE, LOGRM, true>(S, Ws, tid, [&](int n, C v) { return vmul(v, Tv[n]); });
        __syncthreads();
        if (g.nbx > 0) {
            strip_cn<C, T, K::CMAX, N>(S, reinterpret_cast<const C*>(g.cnx), g.nbx, g.blk0x, tid, scan,
                                       [](int, C v) { return v; });
            __syncthreads();
        }
    }
    // rows outside the y- and z-strip blocks take the second V/2 here (CN_y
    // and CN_z are the identity on them); the later passes apply it on the
    // block rows
    const int ry = (int)(y % g.ny1), rz = (int)(y / g.ny1);
    if (MODE == ROW_KVC && g.v2 && ((ry - g.blk0y) & (g.ny1 - 1)) >= g.nby &&
        ((rz - g.blk0z1) & (g.nz1 - 1)) >= g.nbz1) {
#pragma unroll 4
        for (int j = 0; j < E; ++j) {
            const int n = tid + j * T;
            row[n] = vmul(S[swz<C>(n)], Tv[n]);
        }
    } else {
#pragma unroll 4
        for (int j = 0; j < E; ++j) {
            const int n = tid + j * T;
            row[n] = S[swz<C>(n)];
        }
    }
}

// Column pass: TW columns per CTA, each transformed by T = ny/E threads.
// COL_CVK: CN_y on the column's strip block, V/2 (outside the block once the
// tile is loaded, on it as the CN stores), then F_y, e^{-i ky^2 tau/2}/ny,
// F_y^-1; COL_CBK: the same with V/2 on the block rows only (the row pass
// applied the rest); COL_K: the kinetic factor alone.  The last forward
// pass, the factor and the first inverse pass are fused (kcenter; table in
// its transposed order).  The column tile, the V/2 factors of the strip rows
// and the twiddles are staged in shared memory by asynchronous copies issued
// together at the start; the V/2 factors of the other rows and the kinetic
// table (the same for every column) are read through the read-only cache.
template <typename R, int LOGN, int LOGE, int LOGRM, int TW>
struct ColCfg {
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    static constexpr int THREADS = TW * K::T;
    static constexpr int MINB = THREADS >= 512 ? 1 : 512 / THREADS;   // <= 128 registers
    // column pitch: N + 64 bytes, so that the TW columns of one row fall in
    // different banks when the tile is filled and drained row by row
    static constexpr int PITCH = K::N + 64 / (int)sizeof(C);
    using TWT = typename Tw2D<R>::T;
    static constexpr int TWN = TwCountT<TWT, LOGN, LOGRM>::value;
    using VT = typename VabT<R>::T;
    static constexpr size_t OFF_W = sizeof(C) * (size_t)TW * PITCH;
    static constexpr size_t OFF_SCAN = OFF_W + sizeof(TWT) * TWN;
    static constexpr size_t OFF_V = OFF_SCAN + sizeof(C) * 32 * TW;   // scan scratch of each column
    static constexpr int VCAP = K::T * K::CMAX;                       // strip rows a column takes
    static constexpr size_t SMEM_K = OFF_V;
    static constexpr size_t SMEM_CVK = OFF_V + sizeof(VT) * (size_t)TW * VCAP;   // V/2 of the strip rows
    static_assert(OFF_W % 16 == 0 && OFF_SCAN % 16 == 0 && OFF_V % 16 == 0, "16-byte aligned parts");
};

template <typename R, int LOGN, int LOGE, int LOGRM, int TW, int MODE>
__global__ void __launch_bounds__(ColCfg<R, LOGN, LOGE, LOGRM, TW>::THREADS, ColCfg<R, LOGN, LOGE, LOGRM, TW>::MINB)
col_pass_kernel(LineGeo lg, void* __restrict__ psi_v, const void* __restrict__ tky_v)
{
    using CC = ColCfg<R, LOGN, LOGE, LOGRM, TW>;
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    using C = typename K::C;
    using TT = typename K::TT;
    using VT = typename VabT<R>::T;
    using TWT = typename CC::TWT;
    constexpr int N = K::N, T = K::T;
    constexpr int PITCH = CC::PITCH;
    constexpr int NIT = N / T;                      // tile elements per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* S = reinterpret_cast<C*>(smem_raw);
    TWT* Ws = reinterpret_cast<TWT*>(smem_raw + CC::OFF_W);
    const int64_t nx = lg.ld;
    const int64_t gpp = nx / TW;                    // CTAs per plane
    const int64_t poff = (int64_t)(blockIdx.x / gpp) * lg.plane;
    C* __restrict__ psi = reinterpret_cast<C*>(psi_v) + poff;
    const VT* __restrict__ tv = reinterpret_cast<const VT*>(lg.tv) + poff;   // COL_CVK
    const TWT* __restrict__ W = reinterpret_cast<const TWT*>(lg.W);
    const TT* __restrict__ tky = reinterpret_cast<const TT*>(tky_v);
    const int64_t c0 = (int64_t)(blockIdx.x % gpp) * TW;
    VT* Tvs = reinterpret_cast<VT*>(smem_raw + CC::OFF_V);     // [TW][VCAP] (COL_CVK)
#pragma unroll 8
    for (int it = 0; it < NIT; ++it) {              // row by row: the TW columns of a row are adjacent
        const int idx = threadIdx.x + it * TW * T;
        const int yy = idx / TW, j = idx % TW;
        cp_async<sizeof(C)>(&S[j * PITCH + swz<C>(yy)], &psi[(int64_t)yy * nx + c0 + j]);
    }
    if constexpr (MODE == COL_CVK || MODE == COL_CBK) {
        for (int idx = threadIdx.x; idx < lg.nb * TW; idx += TW * T) {
            const int i = idx / TW, j = idx % TW;
            const int yy = (lg.blk0 + i) & (N - 1);
            cp_async<sizeof(VT)>(&Tvs[j * CC::VCAP + i], &tv[(int64_t)yy * nx + c0 + j]);
        }
    }
    for (int i = threadIdx.x; i < CC::TWN; i += TW * T) cp_async<sizeof(TWT)>(&Ws[i], &W[i]);
    cp_async_commit();
    cp_async_wait<0>();
    const int col = threadIdx.x / T, tid = threadIdx.x % T;
    C* Sc = S + col * PITCH;
    bool off_v = MODE == COL_CVK;                    // V/2 off the strip block here
    if (MODE == COL_CVK && lg.sel_div > 0) {
        const int q = (int)((c0 / lg.sel_div) % lg.sel_n);
        off_v = ((q - lg.sel_blk0) & (lg.sel_n - 1)) < lg.sel_nb;
    }
    if (off_v) {
        // V/2 on the thread's own elements outside the strip block (CN along
        // the lines is the identity there; COL_CBK: the row pass applied it)
#pragma unroll 8
        for (int it = 0; it < NIT; ++it) {
            const int idx = threadIdx.x + it * TW * T;
            const int yy = idx / TW, j = idx % TW;
            if (((yy - lg.blk0) & (N - 1)) >= lg.nb) {
                C& v = S[j * PITCH + swz<C>(yy)];
                v = vmul(v, __ldg(&tv[(int64_t)yy * nx + c0 + j]));
            }
        }
    }
    if constexpr (MODE != COL_K) __syncthreads();   // the tile, complete, before the strip CN
    if constexpr (MODE == COL_CVK || MODE == COL_CBK) {
        if (lg.nb > 0) {
            const VT* tvc = Tvs + col * CC::VCAP;
            C* scan = reinterpret_cast<C*>(smem_raw + CC::OFF_SCAN) + 32 * col;
            strip_cn<C, T, K::CMAX, N>(Sc, reinterpret_cast<const C*>(lg.cn), lg.nb, lg.blk0, tid, scan,
                                       [&](int n, C v) { return vmul(v, tvc[(n - lg.blk0) & (N - 1)]); });
        }
    }
    __syncthreads();
    fwd_passes<R, LOGN, LOGE, LOGRM, 0, K::NPASS - 1>(Sc, Ws, tid);
    kcenter<R, LOGN, LOGE, LOGRM>(Sc, tky, tid);
    __syncthreads();
    inv_passes<R, LOGN, LOGE, LOGRM, K::NPASS - 2, 0>(Sc, Ws, tid);
#pragma unroll 8
    for (int it = 0; it < NIT; ++it) {
        const int idx = threadIdx.x + it * TW * T;
        const int yy = idx / TW, j = idx % TW;
        psi[(int64_t)yy * nx + c0 + j] = S[j * PITCH + swz<C>(yy)];
    }
}

// Strip Crank-Nicolson along a strided axis (the 3D step's y-strip pass):
// CN(psi) = 2 M^-1 psi - psi on the block rows of every line, M = LU from
// the host (mf, mb, g).  One thread per line: a CTA stages the block rows of
// TWC adjacent lines (each block row a contiguous segment of TWC elements,
// read and written coalesced) and the coefficients in shared memory, then
// each thread runs the two sweeps of its own line, with no scan and no
// barrier.  The forward sweep leaves y in place of the right-hand side r;
// the backward sweep recovers r_i = y_i - mf_i y_{i-1} from the stored y.
template <typename C, int TWC>
__global__ void __launch_bounds__(TWC)
cn_lines_kernel(CnGeo g, void* __restrict__ psi_v)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nb = g.nb, ny = g.n;
    C* tile = reinterpret_cast<C*>(smem_raw);         // [nb][TWC]
    C* cf = tile + (size_t)nb * TWC;                  // mf, mb, g
    const int64_t nx = g.ld;
    const int64_t gpp = nx / TWC;                     // CTAs per plane
    C* __restrict__ psi = reinterpret_cast<C*>(psi_v) + (int64_t)(blockIdx.x / gpp) * g.plane;
    const C* __restrict__ cn = reinterpret_cast<const C*>(g.cn);
    const int64_t c0 = (int64_t)(blockIdx.x % gpp) * TWC;
    const int t = threadIdx.x;
    for (int i = 0; i < nb; ++i) {
        const int yy = (g.blk0 + i) % ny;
        cp_async<sizeof(C)>(&tile[i * TWC + t], &psi[(int64_t)yy * nx + c0 + t]);
    }
    for (int i = t; i < 3 * nb; i += TWC) cp_async<sizeof(C)>(&cf[i], &cn[i]);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    C y = cmk<C>(0, 0);
    for (int i = 0; i < nb; ++i) {
        y = cfma(cf[i], y, tile[i * TWC + t]);
        tile[i * TWC + t] = y;
    }
    C x = cmk<C>(0, 0);
    for (int i = nb - 1; i >= 0; --i) {
        const C yi = tile[i * TWC + t];
        x = cfma(cf[nb + i], x, cmul(cf[2 * nb + i], yi));
        const C r = i > 0 ? csub(yi, cmul(cf[i], tile[(i - 1) * TWC + t])) : yi;
        tile[i * TWC + t] = cmk<C>(2 * x.x - r.x, 2 * x.y - r.y);
    }
    __syncthreads();
    for (int i = 0; i < nb; ++i) {
        const int yy = (g.blk0 + i) % ny;
        psi[(int64_t)yy * nx + c0 + t] = tile[i * TWC + t];
    }
}

// ---------------------------------------------------------------- launchers
// rows 0 .. nrows-1 (psi == nullptr: set the shared-memory attribute only)
template <typename R, int LOGN, int LOGE, int LOGRM>
int launch_row_t(int mode, const Geo2D& g, void* psi, int nrows, const void* tkx, cudaStream_t st) {
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    const size_t smem = Cfg2DRow<R, LOGN, LOGE, LOGRM>::SMEM2;
    void (*k)(Geo2D, void*, const void*) = nullptr;
    switch (mode) {
    case ROW_K: k = row_pass_kernel<R, LOGN, LOGE, LOGRM, ROW_K>; break;
    case ROW_KVC: k = row_pass_kernel<R, LOGN, LOGE, LOGRM, ROW_KVC>; break;
    default: return SOFT_ERR_INVALID_ARG;
    }
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SOFT_ERR_CUDA;
    if (nrows <= 0 || !psi) return SOFT_OK;
    k<<<nrows, K::T, smem, st>>>(g, psi, tkx);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

// lines of `planes` planes (LineGeo); ld must be a multiple of TW
template <typename R, int LOGN, int LOGE, int LOGRM, int TW>
int launch_col_t(int mode, const LineGeo& g, int planes, void* psi, const void* tky, cudaStream_t st) {
    using CC = ColCfg<R, LOGN, LOGE, LOGRM, TW>;
    using K = Cfg1D<R, LOGN, LOGE, LOGRM>;
    const size_t smem = mode == COL_K ? CC::SMEM_K : CC::SMEM_CVK;
    void (*k)(LineGeo, void*, const void*) = nullptr;
    switch (mode) {
    case COL_K: k = col_pass_kernel<R, LOGN, LOGE, LOGRM, TW, COL_K>; break;
    case COL_CVK: k = col_pass_kernel<R, LOGN, LOGE, LOGRM, TW, COL_CVK>; break;
    case COL_CBK: k = col_pass_kernel<R, LOGN, LOGE, LOGRM, TW, COL_CBK>; break;
    default: return SOFT_ERR_INVALID_ARG;
    }
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SOFT_ERR_CUDA;
    if (!psi) return SOFT_OK;             // attribute set only
    if (g.ld % TW || planes < 1) return SOFT_ERR_INVALID_ARG;
    if (mode != COL_K && (g.nb + K::T - 1) / K::T > K::CMAX) return SOFT_ERR_UNSUPPORTED;
    const int64_t grid = g.ld / TW * planes;
    if (grid > 0x7fffffff) return SOFT_ERR_TOO_LARGE;
    k<<<(unsigned)grid, CC::THREADS, smem, st>>>(g, psi, tky);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

// strip rows of a column pass per thread of the column configuration
template <typename R, int LOGN, int LOGE, int LOGRM>
constexpr int col_strip_capacity() { return Cfg1D<R, LOGN, LOGE, LOGRM>::T * Cfg1D<R, LOGN, LOGE, LOGRM>::CMAX; }

// the strip CN pass: TWC = 128, 64 or 32 lines per CTA, the most whose
// tile fits 100 KB of shared memory (two CTAs per SM), else 32 lines up to
// the 227 KB limit
template <typename C, int TWC>
int launch_cn_lines(const CnGeo& g, int planes, void* psi, size_t smem, cudaStream_t st) {
    auto k = cn_lines_kernel<C, TWC>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SOFT_ERR_CUDA;
    if (!psi) return SOFT_OK;
    const int64_t grid = g.ld / TWC * planes;
    if (grid > 0x7fffffff) return SOFT_ERR_TOO_LARGE;
    k<<<(unsigned)grid, TWC, smem, st>>>(g, psi);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

template <typename C>
int launch_cny_t(const CnGeo& g, int planes, void* psi, cudaStream_t st) {
    if (g.nb <= 0) return SOFT_OK;
    if (planes < 1) return SOFT_ERR_INVALID_ARG;
    auto bytes = [&](int twc) { return sizeof(C) * (size_t)g.nb * (twc + 3); };
    if (g.ld % 128 == 0 && bytes(128) <= 100 * 1024) return launch_cn_lines<C, 128>(g, planes, psi, bytes(128), st);
    if (g.ld % 64 == 0 && bytes(64) <= 100 * 1024) return launch_cn_lines<C, 64>(g, planes, psi, bytes(64), st);
    if (g.ld % 32 == 0 && bytes(32) <= 227 * 1024) return launch_cn_lines<C, 32>(g, planes, psi, bytes(32), st);
    return SOFT_ERR_UNSUPPORTED;
}

}  // namespace soft
