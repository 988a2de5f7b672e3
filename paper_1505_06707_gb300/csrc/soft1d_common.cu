// 1D launch dispatch, the per-call pulse-shape table and the observables
// kernel (norm inside |x| < R0 and the flux through x = +-R0).
#include "soft1d_inst.cuh"

namespace soft {

Launch1D soft1d_c64_a(int logn, int loge, int logrm);
Launch1D soft1d_c64_b(int logn, int loge, int logrm);
Launch1D soft1d_c128_a(int logn, int loge, int logrm);
Launch1D soft1d_c128_b(int logn, int loge, int logrm);

static Launch1D find1d(int prec, int logn, int loge, int logrm) {
    if (prec == SOFT_C64) {
        Launch1D f = soft1d_c64_a(logn, loge, logrm);
        return f ? f : soft1d_c64_b(logn, loge, logrm);
    }
    if (prec == SOFT_C128) {
        Launch1D f = soft1d_c128_a(logn, loge, logrm);
        return f ? f : soft1d_c128_b(logn, loge, logrm);
    }
    return nullptr;
}

bool soft1d_supported(int prec, int logn, int loge, int logrm) {
    return find1d(prec, logn, loge, logrm) != nullptr;
}

// default (elements per thread, largest radix) of each size; the tuner may
// pick another built variant
void soft1d_default_cfg(int prec, int logn, int* loge, int* logrm) {
    int e;
    if (logn <= 6) e = 1;
    else if (logn == 7) e = 2;
    else if (logn <= 9) e = 3;
    else if (prec == SOFT_C64) e = logn >= 13 ? 5 : 4;
    else e = logn >= 14 ? 5 : logn >= 12 ? 4 : 3;   // N = 16384: state in global memory, 512 threads
    *loge = e;
    *logrm = e > 4 ? 4 : e;
    if (prec == SOFT_C128 && *logrm > 3) *logrm = 3;   // radix 16 in FP64 does not fit 128 registers
}

// every built (elements per thread, radix) variant of a size
int soft1d_variants(int prec, int logn, int* loge, int* logrm, int maxv) {
    int k = 0;
    for (int e = 1; e <= 5; ++e)
        for (int r = 1; r <= 4 && r <= e; ++r)
            if (k < maxv && find1d(prec, logn, e, r)) { loge[k] = e; logrm[k] = r; ++k; }
    return k;
}

int launch_soft1d(int prec, int logn, int loge, int logrm, const Inst1D* d_inst, int count,
                  void* psi, int64_t nsteps, const double* ftab, int64_t ftab_stride, int* d_status,
                  cudaStream_t st, size_t* smem_out) {
    Launch1D f = find1d(prec, logn, loge, logrm);
    if (!f) return SOFT_ERR_UNSUPPORTED;
    return f(d_inst, count, psi, nsteps, ftab, ftab_stride, d_status, st, smem_out);
}

// ---------------------------------------------------------------------------
// f_c(s) = sin^2(pi t/Tp) sin(omega t) on [0, Tp], t = t0 + (s + 1/2) tau
__global__ void field_table_kernel(const double* __restrict__ cls, int ncls, double t0, double tau,
                                   int64_t nsteps, double* __restrict__ out, int64_t stride) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (s >= nsteps || c >= ncls) return;
    const double om = cls[2 * c], Tp = cls[2 * c + 1];
    const double t = t0 + ((double)s + 0.5) * tau;
    double v = 0.0;
    if (t >= 0.0 && t <= Tp) {
        const double a = sin(M_PI * t / Tp);
        v = a * a * sin(om * t);
    }
    out[c * stride + s] = v;
}

// the same table with the start time read from device memory (graph replays)
__global__ void field_table_dev_kernel(const double* __restrict__ cls, int ncls,
                                       const double* __restrict__ t0p, double tau, int64_t nsteps,
                                       double* __restrict__ out, int64_t stride) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (s >= nsteps || c >= ncls) return;
    const double om = cls[2 * c], Tp = cls[2 * c + 1];
    const double t = *t0p + ((double)s + 0.5) * tau;
    double v = 0.0;
    if (t >= 0.0 && t <= Tp) {
        const double a = sin(M_PI * t / Tp);
        v = a * a * sin(om * t);
    }
    out[c * stride + s] = v;
}

int launch_field_table_dev(const double* d_cls, int ncls, const double* d_t0, double tau,
                           int64_t nsteps, double* out, int64_t stride, cudaStream_t st) {
    if (ncls <= 0 || nsteps <= 0) return SOFT_OK;
    dim3 grid((unsigned)((nsteps + 255) / 256), (unsigned)ncls);
    field_table_dev_kernel<<<grid, 256, 0, st>>>(d_cls, ncls, d_t0, tau, nsteps, out, stride);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

int launch_field_table(const double* d_cls, int ncls, double t0, double tau, int64_t nsteps,
                       double* out, int64_t stride, cudaStream_t st) {
    if (ncls <= 0 || nsteps <= 0) return SOFT_OK;
    dim3 grid((unsigned)((nsteps + 255) / 256), (unsigned)ncls);
    field_table_kernel<<<grid, 256, 0, st>>>(d_cls, ncls, t0, tau, nsteps, out, stride);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

__global__ void advance_time_kernel(double* t, double dt) { *t += dt; }

int launch_advance_time(double* d_t, double dt, cudaStream_t st) {
    advance_time_kernel<<<1, 1, 0, st>>>(d_t, dt);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

// ---------------------------------------------------------------------------
template <typename C>
__global__ void observe1d_kernel(const Inst1D* __restrict__ insts, const C* __restrict__ psi_base,
                                 double* __restrict__ norm_in, double* __restrict__ flux) {
    const Inst1D I = insts[blockIdx.x];
    const C* psi = psi_base + I.off;
    double acc = 0.0;
    for (int j = I.iL + threadIdx.x; j < I.iR; j += blockDim.x) {
        const double re = (double)psi[j].x, im = (double)psi[j].y;
        acc += re * re + im * im;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        norm_in[blockIdx.x] = tot * I.h;
        const int ia[2] = {I.iL - 1, I.iR - 1};
        for (int e = 0; e < 2; ++e) {
            const int a = (ia[e] + I.n) % I.n, b = (ia[e] + 1) % I.n;
            const double ar = psi[a].x, ai = psi[a].y, br = psi[b].x, bi = psi[b].y;
            const double mr = 0.5 * (ar + br), mi = 0.5 * (ai + bi);
            const double dr = (br - ar) / I.h, di = (bi - ai) / I.h;
            flux[2 * blockIdx.x + e] = mr * di - mi * dr;     // Im(conj(m) d)
        }
    }
}

int launch_observe1d(int prec, const Inst1D* d_inst, int count, const void* psi, double* norm_in,
                     double* flux, cudaStream_t st) {
    if (count <= 0) return SOFT_OK;
    if (prec == SOFT_C64)
        observe1d_kernel<float2><<<count, 256, 0, st>>>(d_inst, (const float2*)psi, norm_in, flux);
    else
        observe1d_kernel<double2><<<count, 256, 0, st>>>(d_inst, (const double2*)psi, norm_in, flux);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

}  // namespace soft
