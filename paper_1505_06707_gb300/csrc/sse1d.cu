// Stationary ECS equation on a 1D grid (Sec. III): A psi = f with
//   A = F^-1 K F + C + U - E            (the matrix under Eq. linsys)
// by complex-symmetric CG with the FFT preconditioner of Eq. PreconFFT or
// the banded ECS preconditioner of Eq. PreconFFT_ECS,
//   P^-1 = F^-1 X^T (Lambda - E)^-1 X F.
//
// One CTA owns one energy for the whole solve: the FFT work buffer and the
// vectors x, r, p, z of that energy stay in shared memory (6 N complex128,
// 192 KB at N = 2048), so an iteration touches global memory only for the
// tables, which every CTA shares through L2.  The scalars of the iteration
// are block sums broadcast through shared memory: every thread takes the
// same branch, and the loop ends at convergence, breakdown or maxit.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "band.h"
#include "pcg.cuh"
#include "plan_internal.h"

namespace soft {

struct Sse1DGeo {
    const double2* W;                  // pass twiddle bases (double2)
    const double2* K;                  // k^2/(2N) in the forward FFT's output order
    const double2* U;                  // U(z(x_j)), natural order
    const double2* C;                  // C[j][j-1], C[j][j], C[j][j+1] (3N)
    int nb, blk0;                      // rows of the cyclic block where C is non-zero
    const int* pos;                    // FFT output position of natural index m
    const int* bs;                     // band start of row nu
    const int* bw;                     // band width of row nu
    const double2* xf;                 // band rows of X (u-major, e^{i k x0}/sqrt N folded in)
    const double2* xb;                 // band rows of X^T (u-major, e^{-i k x0}/sqrt N folded in)
    const double2* lam;                // eigenvalues lambda_nu
};

namespace {

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// sum of v over the CTA, returned to every thread (red: 33 entries)
__device__ __forceinline__ double2 bsum(double2 v, double2* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();                    // red may still be read by the previous sum
    if (l == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0);
        for (int i = 0; i < nw; ++i) { t.x += red[i].x; t.y += red[i].y; }
        red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// w = A p for the CTA's energy (p, w natural order in shared memory; S is
// the swizzled FFT buffer).  Ends with a barrier.
template <int LOGN, int LOGE, int LOGRM>
__device__ __forceinline__ void apply_A(const Sse1DGeo& g, const double2* p, double2* w, double2* S, double En,
                                        int tid) {
    using K = Cfg1D<double, LOGN, LOGE, LOGRM>;
    constexpr int N = K::N, T = K::T, E_ = K::E;
    for (int j = 0; j < E_; ++j) {
        const int n = tid + j * T;
        S[swz<double2>(n)] = p[n];
    }
    __syncthreads();
    fwd_fft<double, LOGN, LOGE, LOGRM, 0>(S, g.W, tid);
    kmul<double, LOGN, LOGE, LOGRM>(S, g.K, tid);
    inv_fft<double, LOGN, LOGE, LOGRM, K::NPASS - 1>(S, g.W, tid);
    for (int j = 0; j < E_; ++j) {
        const int n = tid + j * T;
        const double2 pv = p[n];
        double2 u = __ldg(&g.U[n]);
        u.x -= En;
        double2 v = cfma(u, pv, S[swz<double2>(n)]);
        if (((n - g.blk0) & (N - 1)) < g.nb) {
            v = cfma(__ldg(&g.C[n]), p[(n + N - 1) & (N - 1)], v);
            v = cfma(__ldg(&g.C[N + n]), pv, v);
            v = cfma(__ldg(&g.C[2 * N + n]), p[(n + 1) & (N - 1)], v);
        }
        w[n] = v;
    }
    __syncthreads();
}

// z = P^-1 r (r, z natural order; T1 natural-order scratch; S the FFT
// buffer).  The paper's F has e^{+ikx}: conj(FFT(conj(.))).  Ends with a barrier.
template <int LOGN, int LOGE, int LOGRM>
__device__ __forceinline__ void apply_P(const Sse1DGeo& g, const double2* r, double2* z, double2* S, double2* T1,
                                        double En, int tid) {
    using K = Cfg1D<double, LOGN, LOGE, LOGRM>;
    constexpr int N = K::N, T = K::T, E_ = K::E;
    for (int j = 0; j < E_; ++j) {
        const int n = tid + j * T;
        S[swz<double2>(n)] = cconj(r[n]);
    }
    __syncthreads();
    fwd_fft<double, LOGN, LOGE, LOGRM, 0>(S, g.W, tid);
    for (int j = 0; j < E_; ++j) {
        const int m = tid + j * T;
        T1[m] = cconj(S[swz<double2>(__ldg(&g.pos[m]))]);
    }
    __syncthreads();
    for (int j = 0; j < E_; ++j) {               // X F r, then / (lambda - E)
        const int nu = tid + j * T;
        const int s0 = __ldg(&g.bs[nu]), wd = __ldg(&g.bw[nu]);
        double2 o = make_double2(0.0, 0.0);
        for (int u = 0; u < wd; ++u) o = cfma(__ldg(&g.xf[u * N + nu]), T1[s0 + u], o);
        double2 den = __ldg(&g.lam[nu]);
        den.x -= En;
        z[nu] = cdiv(o, den);
    }
    __syncthreads();
    for (int j = 0; j < E_; ++j) {               // X^T into the FFT positions (conjugated)
        const int m = tid + j * T;
        const int s0 = __ldg(&g.bs[m]), wd = __ldg(&g.bw[m]);
        double2 o = make_double2(0.0, 0.0);
        for (int u = 0; u < wd; ++u) o = cfma(__ldg(&g.xb[u * N + m]), z[s0 + u], o);
        S[swz<double2>(__ldg(&g.pos[m]))] = cconj(o);
    }
    __syncthreads();
    inv_fft<double, LOGN, LOGE, LOGRM, K::NPASS - 1>(S, g.W, tid);
    for (int j = 0; j < E_; ++j) {
        const int n = tid + j * T;
        z[n] = cconj(S[swz<double2>(n)]);
    }
    __syncthreads();
}

template <int LOGN, int LOGE, int LOGRM>
constexpr size_t sse1d_smem() {
    return sizeof(double2) * (6 * (size_t(1) << LOGN) + 33);
}

// COCG (Sec. III after Eq. linsys: the bilinear r^T z replaces the inner
// product), x0 = 0, stop when ||r||_2/||f||_2 < tol; energy blockIdx.x
template <int LOGN, int LOGE, int LOGRM>
__global__ void __launch_bounds__(Cfg1D<double, LOGN, LOGE, LOGRM>::T, 1)
sse1d_cocg_kernel(Sse1DGeo g, const double2* __restrict__ f, double2* __restrict__ xout,
                  const double* __restrict__ Es, double tol, int maxit, int* __restrict__ iters,
                  double* __restrict__ relres, int* __restrict__ status)
{
    using K = Cfg1D<double, LOGN, LOGE, LOGRM>;
    constexpr int N = K::N, T = K::T, E_ = K::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* S = reinterpret_cast<double2*>(smem_raw);
    double2* T1 = S + N;
    double2* x = T1 + N;
    double2* r = x + N;
    double2* p = r + N;
    double2* z = p + N;
    double2* red = z + N;
    const int e = blockIdx.x, tid = threadIdx.x;
    const double En = Es[e];
    double ff = 0.0;
    for (int j = 0; j < E_; ++j) {
        const int n = tid + j * T;
        const double2 fv = f[n];
        r[n] = fv;
        x[n] = make_double2(0.0, 0.0);
        ff += fv.x * fv.x + fv.y * fv.y;
    }
    ff = bsum(make_double2(ff, 0.0), red).x;
    int st = SOFT_ERR_NOT_CONVERGED, it = 0;
    double rel = 1.0;
    if (!(ff > 0.0) || !isfinite(ff)) {
        st = ff == 0.0 ? SOFT_OK : SOFT_ERR_NONFINITE;
        rel = 0.0;
    } else {
        apply_P<LOGN, LOGE, LOGRM>(g, r, z, S, T1, En, tid);
        double2 acc = make_double2(0.0, 0.0);
        for (int j = 0; j < E_; ++j) {
            const int n = tid + j * T;
            p[n] = z[n];
            acc = cfma(r[n], z[n], acc);
        }
        double2 rho = bsum(acc, red);
        while (it < maxit) {
            apply_A<LOGN, LOGE, LOGRM>(g, p, T1, S, En, tid);          // w = A p in T1
            acc = make_double2(0.0, 0.0);
            for (int j = 0; j < E_; ++j) {
                const int n = tid + j * T;
                acc = cfma(p[n], T1[n], acc);
            }
            const double2 pw = bsum(acc, red);
            if (!(pw.x * pw.x + pw.y * pw.y > 0.0)) { st = SOFT_ERR_BREAKDOWN; break; }
            const double2 al = cdiv(rho, pw);
            double rr = 0.0;
            for (int j = 0; j < E_; ++j) {
                const int n = tid + j * T;
                x[n] = cfma(al, p[n], x[n]);
                const double2 rv = csub(r[n], cmul(al, T1[n]));
                r[n] = rv;
                rr += rv.x * rv.x + rv.y * rv.y;
            }
            rr = bsum(make_double2(rr, 0.0), red).x;
            ++it;
            rel = sqrt(rr / ff);
            if (!isfinite(rel)) { st = SOFT_ERR_NONFINITE; break; }
            if (rel < tol) { st = SOFT_OK; break; }
            apply_P<LOGN, LOGE, LOGRM>(g, r, z, S, T1, En, tid);
            acc = make_double2(0.0, 0.0);
            for (int j = 0; j < E_; ++j) {
                const int n = tid + j * T;
                acc = cfma(r[n], z[n], acc);
            }
            const double2 rn = bsum(acc, red);
            if (!(rho.x * rho.x + rho.y * rho.y > 0.0)) { st = SOFT_ERR_BREAKDOWN; break; }
            const double2 be = cdiv(rn, rho);
            rho = rn;
            for (int j = 0; j < E_; ++j) {
                const int n = tid + j * T;
                p[n] = cfma(be, p[n], z[n]);
            }
            __syncthreads();
        }
    }
    for (int j = 0; j < E_; ++j) {
        const int n = tid + j * T;
        xout[(int64_t)e * N + n] = x[n];
    }
    if (tid == 0) {
        iters[e] = it;
        relres[e] = rel;
        status[e] = st;
    }
}

// one application: what = 0: y = A x; 1: y = P^-1 x
template <int LOGN, int LOGE, int LOGRM>
__global__ void __launch_bounds__(Cfg1D<double, LOGN, LOGE, LOGRM>::T, 1)
sse1d_apply_kernel(Sse1DGeo g, const double2* __restrict__ in, double2* __restrict__ out, double En, int what)
{
    using K = Cfg1D<double, LOGN, LOGE, LOGRM>;
    constexpr int N = K::N, T = K::T, E_ = K::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* S = reinterpret_cast<double2*>(smem_raw);
    double2* T1 = S + N;
    double2* a = T1 + N;
    double2* b = a + N;
    const int tid = threadIdx.x;
    for (int j = 0; j < E_; ++j) a[tid + j * T] = in[tid + j * T];
    __syncthreads();
    if (what == 0) apply_A<LOGN, LOGE, LOGRM>(g, a, b, S, En, tid);
    else apply_P<LOGN, LOGE, LOGRM>(g, a, b, S, T1, En, tid);
    for (int j = 0; j < E_; ++j) out[tid + j * T] = b[tid + j * T];
}

template <int LOGN, int LOGE, int LOGRM>
int launch_t(const Sse1DGeo& g, int mode, const double2* in, double2* out, const double* dE, double En, int nE,
             double tol, int maxit, int* iters, double* relres, int* status, cudaStream_t st) {
    using K = Cfg1D<double, LOGN, LOGE, LOGRM>;
    const size_t smem = sse1d_smem<LOGN, LOGE, LOGRM>();
    static_assert(sse1d_smem<LOGN, LOGE, LOGRM>() <= 227 * 1024, "shared memory");
    if (mode == 0) {
        auto k = sse1d_cocg_kernel<LOGN, LOGE, LOGRM>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return SOFT_ERR_CUDA;
        if (nE > 0) k<<<nE, K::T, smem, st>>>(g, in, out, dE, tol, maxit, iters, relres, status);
    } else {
        auto k = sse1d_apply_kernel<LOGN, LOGE, LOGRM>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return SOFT_ERR_CUDA;
        k<<<1, K::T, smem, st>>>(g, in, out, En, mode - 1);
    }
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

// the FFT configuration of each supported size (E a multiple of 4, radix 8)
bool cfg_for(int logn, int* loge, int* logrm) {
    if (logn < 8 || logn > 11) return false;
    *loge = 3;
    *logrm = 3;
    return true;
}

int launch(int logn, const Sse1DGeo& g, int mode, const double2* in, double2* out, const double* dE, double En,
           int nE, double tol, int maxit, int* iters, double* relres, int* status, cudaStream_t st) {
    switch (logn) {
    case 8: return launch_t<8, 3, 3>(g, mode, in, out, dE, En, nE, tol, maxit, iters, relres, status, st);
    case 9: return launch_t<9, 3, 3>(g, mode, in, out, dE, En, nE, tol, maxit, iters, relres, status, st);
    case 10: return launch_t<10, 3, 3>(g, mode, in, out, dE, En, nE, tol, maxit, iters, relres, status, st);
    case 11: return launch_t<11, 3, 3>(g, mode, in, out, dE, En, nE, tol, maxit, iters, relres, status, st);
    }
    return SOFT_ERR_UNSUPPORTED;
}

}  // namespace

// Per-plan tables of the 1D solver, built on first use.
struct Sse1D {
    int logn = 0, loge = 0, logrm = 0, n = 0;
    void *W = nullptr, *K = nullptr, *U = nullptr, *C = nullptr, *pos = nullptr;
    void* pc[2][5] = {};               // per preconditioner: bs, bw, xf, xb, lam
    double* dE = nullptr;
    int* iters = nullptr;
    double* relres = nullptr;
    int* status = nullptr;
    int cap = 0;
    Sse1DGeo geo[2] = {};
    ~Sse1D() {
        cudaFree(W); cudaFree(K); cudaFree(U); cudaFree(C); cudaFree(pos);
        for (auto& t : pc)
            for (void* b : t) cudaFree(b);
        cudaFree(dE); cudaFree(iters); cudaFree(relres); cudaFree(status);
    }
};

void sse1d_free(Sse1D* s) { delete s; }

static int upload_int(void** dst, const std::vector<int>& v) {
    return upload(dst, v.data(), v.size() * sizeof(int));
}

static int build(soft_plan* P) {
    if (P->s1) return SOFT_OK;
    const Tables1D& TB = *P->tabs[0];
    std::unique_ptr<Sse1D> S(new Sse1D());
    S->n = TB.ax.n;
    S->logn = TB.logn;
    if (!cfg_for(S->logn, &S->loge, &S->logrm)) return SOFT_ERR_UNSUPPORTED;
    const Axis1D& A = TB.ax;
    const int n = S->n;
    int rc;
    if ((rc = upload_c(&S->W, pass_twiddles(S->logn, S->logrm), SOFT_C128))) return rc;
    const std::vector<int> perm = dif_output_order(S->logn, S->logrm);
    std::vector<cd> kt(n);
    std::vector<int> pos(n);
    for (int q = 0; q < n; ++q) {
        kt[q] = 0.5 * A.k[perm[q]] * A.k[perm[q]] / n;
        pos[perm[q]] = q;
    }
    if ((rc = upload_c(&S->K, kt, SOFT_C128))) return rc;
    if ((rc = upload_int(&S->pos, pos))) return rc;
    if ((rc = upload_c(&S->U, TB.U0, SOFT_C128))) return rc;
    std::vector<cd> c = A.Cs;
    c.insert(c.end(), A.Cd.begin(), A.Cd.end());
    c.insert(c.end(), A.Cu.begin(), A.Cu.end());
    if ((rc = upload_c(&S->C, c, SOFT_C128))) return rc;
    for (int type = 0; type < 2; ++type) {
        BandAxis B;
        double chk = 0;
        if ((rc = build_band_axis(A, P->opt.band_width, type == 0, B, &chk))) return rc;
        int wmax = 1;
        for (int wd : B.width) wmax = std::max(wmax, wd);
        std::vector<cd> xf((size_t)wmax * n, 0.0), xb((size_t)wmax * n, 0.0);
        for (int nu = 0; nu < n; ++nu)
            for (int u = 0; u < B.width[nu]; ++u) {
                xf[(size_t)u * n + nu] = B.xf[(size_t)B.off[nu] + u];
                xb[(size_t)u * n + nu] = B.xb[(size_t)B.off[nu] + u];
            }
        void** t = S->pc[type];
        if ((rc = upload_int(&t[0], B.start))) return rc;
        if ((rc = upload_int(&t[1], B.width))) return rc;
        if ((rc = upload_c(&t[2], xf, SOFT_C128))) return rc;
        if ((rc = upload_c(&t[3], xb, SOFT_C128))) return rc;
        if ((rc = upload_c(&t[4], B.lam, SOFT_C128))) return rc;
        Sse1DGeo& g = S->geo[type];
        g.W = (const double2*)S->W; g.K = (const double2*)S->K; g.U = (const double2*)S->U;
        g.C = (const double2*)S->C; g.nb = TB.nb; g.blk0 = TB.blk0; g.pos = (const int*)S->pos;
        g.bs = (const int*)t[0]; g.bw = (const int*)t[1]; g.xf = (const double2*)t[2];
        g.xb = (const double2*)t[3]; g.lam = (const double2*)t[4];
    }
    P->s1 = S.release();
    return SOFT_OK;
}

static bool usable(const soft_plan* P) {
    return P && P->kind == 1 && P->single && P->tabs.size() == 1;
}

int sse1d_refill_potential(soft_plan* P) {
    if (!P->s1) return SOFT_OK;
    return refill_c(P->s1->U, P->tabs[0]->U0, SOFT_C128);
}

int sse1d_solve(soft_plan* P, const double* E, int nE, const void* rhs, void* psi_out, double tol, int maxit,
                int precond, int* iters_out, double* relres_out, cudaStream_t st) {
    if (!usable(P)) return SOFT_ERR_INVALID_ARG;
    if (precond != 0 && precond != 1) return SOFT_ERR_UNSUPPORTED;
    if (P->prec != SOFT_C128) return SOFT_ERR_UNSUPPORTED;
    int rc = build(P);
    if (rc) return rc;
    Sse1D* S = P->s1;
    if (S->cap < nE) {
        cudaFree(S->dE); cudaFree(S->iters); cudaFree(S->relres); cudaFree(S->status);
        S->dE = nullptr; S->iters = nullptr; S->relres = nullptr; S->status = nullptr; S->cap = 0;
        if ((rc = cuda_status(cudaMalloc((void**)&S->dE, sizeof(double) * nE)))) return rc;
        if ((rc = cuda_status(cudaMalloc((void**)&S->iters, sizeof(int) * nE)))) return rc;
        if ((rc = cuda_status(cudaMalloc((void**)&S->relres, sizeof(double) * nE)))) return rc;
        if ((rc = cuda_status(cudaMalloc((void**)&S->status, sizeof(int) * nE)))) return rc;
        S->cap = nE;
    }
    // pageable source: staged before cudaMemcpyAsync returns
    if ((rc = cuda_status(cudaMemcpyAsync(S->dE, E, sizeof(double) * nE, cudaMemcpyHostToDevice, st)))) return rc;
    if ((rc = launch(S->logn, S->geo[precond], 0, (const double2*)rhs, (double2*)psi_out, S->dE, 0.0, nE, tol,
                     maxit, S->iters, S->relres, S->status, st)))
        return rc;
    P->last_launches = 1;
    std::vector<int> it(nE), stt(nE);
    std::vector<double> rr(nE);
    if ((rc = cuda_status(cudaMemcpyAsync(it.data(), S->iters, sizeof(int) * nE, cudaMemcpyDeviceToHost, st)))) return rc;
    if ((rc = cuda_status(cudaMemcpyAsync(rr.data(), S->relres, sizeof(double) * nE, cudaMemcpyDeviceToHost, st)))) return rc;
    if ((rc = cuda_status(cudaMemcpyAsync(stt.data(), S->status, sizeof(int) * nE, cudaMemcpyDeviceToHost, st)))) return rc;
    if ((rc = cuda_status(cudaStreamSynchronize(st)))) return rc;
    if (iters_out) std::memcpy(iters_out, it.data(), sizeof(int) * nE);
    if (relres_out) std::memcpy(relres_out, rr.data(), sizeof(double) * nE);
    int out = SOFT_OK;
    for (int e = 0; e < nE; ++e) {
        if (stt[e] == SOFT_ERR_BREAKDOWN || stt[e] == SOFT_ERR_NONFINITE) return stt[e];
        if (stt[e] != SOFT_OK) out = SOFT_ERR_NOT_CONVERGED;
    }
    return out;
}

int sse1d_apply(soft_plan* P, double E, int what, int precond, const void* x, void* y, cudaStream_t st) {
    if (!usable(P)) return SOFT_ERR_INVALID_ARG;
    if (what == 1 && precond != 0 && precond != 1) return SOFT_ERR_UNSUPPORTED;
    if (P->prec != SOFT_C128) return SOFT_ERR_UNSUPPORTED;
    int rc = build(P);
    if (rc) return rc;
    Sse1D* S = P->s1;
    P->last_launches = 1;
    return launch(S->logn, S->geo[what == 1 ? precond : 0], what == 0 ? 1 : 2, (const double2*)x, (double2*)y,
                  nullptr, E, 1, 0.0, 0, nullptr, nullptr, nullptr, st);
}

}  // namespace soft
