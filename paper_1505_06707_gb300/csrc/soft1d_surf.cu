// Amplitude extraction of the paper's test (Sec. I and Sec. IV: t&E-SURFF)
// on a single 1D complex128 plan:
//   - soft_step_surface: the 1D step with psi and dpsi/dx sampled at the two
//     boundaries x = +-R0 of the unscaled region after every step, fused
//     into the k-space stage of the step kernel (the trigonometric
//     interpolant of the grid function, evaluated from the spectrum the
//     kernel already holds);
//   - sse_surff: the momentum amplitudes A(+-k), k = sqrt(2E), from the
//     time integral of the surface flux (Simpson or Filon-Simpson) and the
//     surface values of the stationary solutions with right-hand side
//     psi(t_max) (E-SURFF), one CTA per energy.
// For a packet that is free beyond R0, with plane waves
// chi_k = (2 pi)^-1/2 e^{ikx - iEt}:
//   A(k) = -/+ (i/2) (2 pi)^-1/2 e^{-ik xs} [ int e^{iEt} (psi' + ik psi)(xs, t) dt
//                                             + i e^{iET} (phi' + ik phi)(xs) ],
// xs = +R0 for k > 0 (sign -), -R0 for k < 0 (sign +), (E - H) phi = psi(T).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "plan_internal.h"
#include "soft1d.cuh"

namespace soft {

namespace {

using SurfLaunch = int (*)(const Inst1D*, void*, int64_t, const double*, int64_t, int*, const void*, void*,
                           cudaStream_t);

// the sampled step kernel is built for the default complex128 configuration
// of N = 256 .. 8192
SurfLaunch find_surf(int logn, int loge, int logrm) {
#define SURF_CASE(LN, LE, LRM) \
    if (logn == LN && loge == LE && logrm == LRM) return &launch_soft1d_surf_t<double, LN, LE, LRM>;
    SURF_CASE(8, 3, 3) SURF_CASE(9, 3, 3) SURF_CASE(10, 3, 3) SURF_CASE(11, 3, 3)
    SURF_CASE(12, 4, 3) SURF_CASE(13, 4, 3)
#undef SURF_CASE
    return nullptr;
}

struct SurfTabs {
    void* sw = nullptr;      // 8 rows x N: the kernel's spectral weights (two sets)
    void* xw = nullptr;      // 4 rows x N: x-space weights of the same interpolant
    ~SurfTabs() { cudaFree(sw); cudaFree(xw); }
};

// Host FP64 tables of the interpolant psi(x) = (1/N) sum_f c_f e^{i k_f (x - x_0)},
// c = DFT(psi) (e^{-2 pi i f j/N}), at x = +R0 and -R0 (rows: psi(R0),
// psi'(R0), psi(-R0), psi'(-R0)).
int build_surf(soft_plan* P, SurfTabs* S) {
    const Tables1D& T = *P->tabs[0];
    const Axis1D& A = T.ax;
    const int n = A.n, logn = T.logn;
    const double x0 = A.x[0], R = T.R0, tau = P->dt;
    const std::vector<int> perm = dif_output_order(logn, T.logrm);
    const int lrl = (logn % T.logrm) ? logn % T.logrm : T.logrm;
    const int Rl = 1 << lrl, nbf = n >> lrl;
    std::vector<cd> sw((size_t)8 * n), xw((size_t)4 * n);
    const double xs[2] = {R, -R};
    for (int p = 0; p < n; ++p) {
        const double k = A.k[perm[p]];
        const int q = (p % Rl) * nbf + p / Rl;       // the kernel's transposed index
        const cd half = std::polar(1.0, -0.25 * k * k * tau);
        for (int side = 0; side < 2; ++side) {
            const cd e = std::polar(1.0 / n, k * (xs[side] - x0));
            const cd d = cd(0.0, k) * e;
            sw[(size_t)(2 * side) * n + q] = e;
            sw[(size_t)(2 * side + 1) * n + q] = d;
            sw[(size_t)(4 + 2 * side) * n + q] = e * half;
            sw[(size_t)(5 + 2 * side) * n + q] = d * half;
        }
    }
    // x-space rows: w_r[j] = (1/N) sum_f a_r(f) e^{-2 pi i f j/N}
    std::vector<cd> root(n);
    for (int m = 0; m < n; ++m) root[m] = std::polar(1.0, -2.0 * 3.14159265358979323846 * m / n);
    for (int side = 0; side < 2; ++side) {
        std::vector<cd> a(n), b(n);
        for (int f = 0; f < n; ++f) {
            a[f] = std::polar(1.0 / n, A.k[f] * (xs[side] - x0));
            b[f] = cd(0.0, A.k[f]) * a[f];
        }
        for (int j = 0; j < n; ++j) {
            cd s0 = 0.0, s1 = 0.0;
            for (int f = 0; f < n; ++f) {
                const cd w = root[(int)(((int64_t)f * j) % n)];
                s0 += a[f] * w;
                s1 += b[f] * w;
            }
            xw[(size_t)(2 * side) * n + j] = s0;
            xw[(size_t)(2 * side + 1) * n + j] = s1;
        }
    }
    int rc;
    if ((rc = upload_c(&S->sw, sw, SOFT_C128))) return rc;
    return upload_c(&S->xw, xw, SOFT_C128);
}

__device__ __forceinline__ double2 cexpi(double ph) {
    double s, c;
    sincos(ph, &s, &c);
    return make_double2(c, s);
}

__device__ __forceinline__ double2 bsum2(double2 v, double2* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
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

// int_{-tau}^{tau} e^{i w u} u^p du, p = 0, 1, 2, th = w tau (series for small |th|)
__device__ void panel_moments(double th, double tau, double2* m) {
    if (fabs(th) < 1e-3) {
        const double t2 = th * th;
        m[0] = make_double2(2 * tau * (1 - t2 / 6 + t2 * t2 / 120), 0.0);
        m[1] = make_double2(0.0, 2 * tau * tau * th * (1.0 / 3 - t2 / 30));
        m[2] = make_double2(2 * tau * tau * tau * (1.0 / 3 - t2 / 10 + t2 * t2 / 168), 0.0);
        return;
    }
    double s, c;
    sincos(th, &s, &c);
    const double w = th / tau;
    m[0] = make_double2(2 * s / w, 0.0);
    m[1] = make_double2(0.0, 2 * (s - th * c) / (w * w));
    m[2] = make_double2(2 * ((th * th - 2) * s + 2 * th * c) / (w * w * w), 0.0);
}

// one CTA per energy: out[2e] = A(+k), out[2e + 1] = A(-k)
__global__ void __launch_bounds__(256)
surff_kernel(const double2* __restrict__ xw, int n, const double2* __restrict__ phi,
             const double2* __restrict__ samp, int64_t ns, double t0, double tau, double R,
             const double* __restrict__ Es, int rule, double2* __restrict__ out)
{
    __shared__ double2 red[33];
    const int e = blockIdx.x, tid = threadIdx.x;
    const double E = Es[e], k = sqrt(2.0 * E), T = t0 + tau * (double)(ns - 1);
    // surface values of phi_E = -phi (A phi = psi(T), A = H - E)
    double2 pv[4];
    const double2* ph = phi + (int64_t)e * n;
    for (int r = 0; r < 4; ++r) {
        double2 a = make_double2(0.0, 0.0);
        for (int j = tid; j < n; j += blockDim.x) a = cfma(__ldg(&xw[(int64_t)r * n + j]), ph[j], a);
        const double2 s = bsum2(a, red);
        pv[r] = make_double2(-s.x, -s.y);
    }
    // time integrals of e^{iEt} (psi' + i kk psi)(xs, t), kk = +k (right), -k (left)
    double2 I[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    double2 mom[3];
    panel_moments(E * tau, tau, mom);
    const int64_t npan = (ns - 1) / 2;
    if (rule == 0) {
        for (int64_t s = tid; s < ns; s += blockDim.x) {
            const double wgt = (s == 0 || s == ns - 1) ? 1.0 : ((s & 1) ? 4.0 : 2.0);
            const double2 ex = cexpi(E * (t0 + tau * (double)s));
            for (int side = 0; side < 2; ++side) {
                const double kk = side ? -k : k;
                const double2 p0 = samp[4 * s + 2 * side], p1 = samp[4 * s + 2 * side + 1];
                const double2 g = make_double2(p1.x - kk * p0.y, p1.y + kk * p0.x);
                I[side] = cfma(cscale(ex, wgt * tau / 3.0), g, I[side]);
            }
        }
    } else {
        for (int64_t j = tid; j < npan; j += blockDim.x) {
            const int64_t s0 = 2 * j;
            const double2 ex = cexpi(E * (t0 + tau * (double)(s0 + 1)));
            for (int side = 0; side < 2; ++side) {
                const double kk = side ? -k : k;
                double2 g[3];
                for (int q = 0; q < 3; ++q) {
                    const double2 p0 = samp[4 * (s0 + q) + 2 * side], p1 = samp[4 * (s0 + q) + 2 * side + 1];
                    g[q] = make_double2(p1.x - kk * p0.y, p1.y + kk * p0.x);
                }
                const double2 a = g[1];
                const double2 b = cscale(csub(g[2], g[0]), 0.5 / tau);
                const double2 c = cscale(cadd(csub(g[2], cscale(g[1], 2.0)), g[0]), 0.5 / (tau * tau));
                const double2 pan = cfma(c, mom[2], cfma(b, mom[1], cmul(a, mom[0])));
                I[side] = cfma(ex, pan, I[side]);
            }
        }
    }
    I[0] = bsum2(I[0], red);
    I[1] = bsum2(I[1], red);
    if (tid == 0) {
        const double pre = 0.5 / sqrt(2.0 * 3.14159265358979323846);
        const double2 eT = cexpi(E * T);
        for (int side = 0; side < 2; ++side) {
            const double kk = side ? -k : k, xs = side ? -R : R, sg = side ? 1.0 : -1.0;
            const double2 D = make_double2(pv[2 * side + 1].x - kk * pv[2 * side].y,
                                           pv[2 * side + 1].y + kk * pv[2 * side].x);
            const double2 iD = cmul(make_double2(0.0, 1.0), cmul(eT, D));
            const double2 tot = cadd(I[side], iD);
            // sg * (i/2) (2 pi)^-1/2 e^{-i kk xs} tot
            const double2 f = cmul(make_double2(0.0, sg * pre), cexpi(-kk * xs));
            out[2 * e + side] = cmul(f, tot);
        }
    }
}

}  // namespace

struct Surf1D {
    SurfTabs t;
    double* dE = nullptr;
    int cap = 0;
    ~Surf1D() { cudaFree(dE); }
};

void surf1d_free(Surf1D* s) { delete s; }

static int ensure_surf(soft_plan* P) {
    if (P->sf) return SOFT_OK;
    std::unique_ptr<Surf1D> S(new Surf1D());
    int rc = build_surf(P, &S->t);
    if (rc) return rc;
    P->sf = S.release();
    return SOFT_OK;
}

static bool surf_plan(const soft_plan* P) {
    return P && P->kind == 1 && P->single && P->tabs.size() == 1 && P->groups.size() == 1 &&
           P->prec == SOFT_C128;
}

}  // namespace soft

using namespace soft;

static int soft_step_surface_impl(soft_plan* P, void* psi, int64_t nsteps, const soft_field* field,
                                             double* t_inout, void* samples, void* stream) {
    if (!P || !psi || !t_inout || !samples || nsteps < 0) return SOFT_ERR_INVALID_ARG;
    if (!surf_plan(P)) return SOFT_ERR_UNSUPPORTED;
    const Group1D& g = P->groups[0];
    SurfLaunch f = find_surf(g.logn, g.loge, g.logrm);
    if (!f) return SOFT_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = P->set_single_field(field, st);
    if (rc) return rc;
    if ((rc = ensure_surf(P))) return rc;
    P->last_launches = 0;
    if (nsteps == 0) return SOFT_OK;
    const double t0 = *t_inout;
    const bool fld = P->inst[0].has_field;
    double2* out = static_cast<double2*>(samples);
    int64_t done = 0;
    while (done < nsteps) {
        const int64_t chunk = std::min<int64_t>(P->ftab_cap, nsteps - done);
        const double tc = t0 + (double)done * P->dt;
        if (fld) {
            if ((rc = launch_field_table(P->d_cls, P->ncls + 1, tc, P->dt, chunk, P->d_ftab, P->ftab_cap, st)))
                return rc;
            ++P->last_launches;
        }
        // the chunk writes samples done .. done + chunk (its first row repeats
        // the previous chunk's last, with the same value)
        if ((rc = f(g.d_inst, psi, chunk, P->d_ftab, P->ftab_cap, P->d_status, P->sf->t.sw, out + 4 * done, st)))
            return rc;
        ++P->last_launches;
        done += chunk;
    }
    *t_inout = t0 + (double)nsteps * P->dt;
    return SOFT_OK;
}
extern "C" int soft_step_surface(soft_plan* P, void* psi, int64_t nsteps, const soft_field* field,
                                 double* t_inout, void* samples, void* stream) {
    return abi_guard([&] { return soft_step_surface_impl(P, psi, nsteps, field, t_inout, samples, stream); });
}

static int sse_surff_impl(soft_plan* P, int nE, const double* E, const void* phi, const void* samples,
                                     int64_t nsamples, double t0, int rule, void* amp, void* stream) {
    if (!P || nE <= 0 || !E || !phi || !samples || !amp || nsamples < 3 || (nsamples - 1) % 2)
        return SOFT_ERR_INVALID_ARG;
    if (rule != 0 && rule != 1) return SOFT_ERR_INVALID_ARG;
    for (int e = 0; e < nE; ++e)
        if (!(E[e] > 0) || !std::isfinite(E[e])) return SOFT_ERR_INVALID_ARG;
    if (!surf_plan(P)) return SOFT_ERR_UNSUPPORTED;
    int rc = ensure_surf(P);
    if (rc) return rc;
    Surf1D* S = P->sf;
    cudaStream_t st = (cudaStream_t)stream;
    if (S->cap < nE) {
        cudaFree(S->dE);
        S->dE = nullptr;
        S->cap = 0;
        if ((rc = cuda_status(cudaMalloc((void**)&S->dE, sizeof(double) * nE)))) return rc;
        S->cap = nE;
    }
    if ((rc = cuda_status(cudaMemcpyAsync(S->dE, E, sizeof(double) * nE, cudaMemcpyHostToDevice, st)))) return rc;
    const Tables1D& T = *P->tabs[0];
    surff_kernel<<<nE, 256, 0, st>>>((const double2*)S->t.xw, T.ax.n, (const double2*)phi,
                                     (const double2*)samples, nsamples, t0, P->dt, T.R0, S->dE, rule,
                                     (double2*)amp);
    P->last_launches = 1;
    return cuda_status(cudaGetLastError());
}
extern "C" int sse_surff(soft_plan* P, int nE, const double* E, const void* phi, const void* samples,
                         int64_t nsamples, double t0, int rule, void* amp, void* stream) {
    return abi_guard([&] { return sse_surff_impl(P, nE, E, phi, samples, nsamples, t0, rule, amp, stream); });
}
