// C ABI of the library: plan construction (host FP64 tables, uploaded once)
// and the 1D step / observables entry points.  The 2D and stationary entry
// points live in plan2d.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "nn.h"
#include "plan_internal.h"

using namespace soft;

namespace soft {

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SOFT_OK;
    if (e == cudaErrorMemoryAllocation) return SOFT_ERR_OOM;
    return SOFT_ERR_CUDA;
}

int upload(void** dst, const void* src, size_t bytes) {
    if (bytes == 0) { *dst = nullptr; return SOFT_OK; }
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) { *dst = nullptr; return cuda_status(e); }
    e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    return cuda_status(e);
}

// phase table: double2 for complex128 plans; (hi, lo) float4 for complex64 plans
int upload_tab(void** dst, const std::vector<cd>& v, int prec) {
    if (prec == SOFT_C128) return upload_c(dst, v, prec);
    std::vector<float> buf(4 * v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        const float hr = (float)v[i].real(), hi = (float)v[i].imag();
        buf[4 * i] = hr;
        buf[4 * i + 1] = hi;
        buf[4 * i + 2] = (float)(v[i].real() - (double)hr);
        buf[4 * i + 3] = (float)(v[i].imag() - (double)hi);
    }
    return upload(dst, buf.data(), buf.size() * sizeof(float));
}

// potential factor table: the factor itself (double2) for complex128 plans;
// its difference from 1 (float2) for complex64 plans
int upload_vtab(void** dst, const std::vector<cd>& v, int prec) {
    if (prec == SOFT_C128) return upload_c(dst, v, prec);
    std::vector<float> buf(2 * v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        buf[2 * i] = (float)(v[i].real() - 1.0);
        buf[2 * i + 1] = (float)v[i].imag();
    }
    return upload(dst, buf.data(), buf.size() * sizeof(float));
}

// round a complex FP64 vector to the plan precision and upload it
int upload_c(void** dst, const std::vector<cd>& v, int prec) {
    if (prec == SOFT_C128) {
        std::vector<double> buf(2 * v.size());
        for (size_t i = 0; i < v.size(); ++i) { buf[2 * i] = v[i].real(); buf[2 * i + 1] = v[i].imag(); }
        return upload(dst, buf.data(), buf.size() * sizeof(double));
    }
    std::vector<float> buf(2 * v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        buf[2 * i] = (float)v[i].real();
        buf[2 * i + 1] = (float)v[i].imag();
    }
    return upload(dst, buf.data(), buf.size() * sizeof(float));
}

// FFT twiddle table (unit-modulus values): complex128 as is; complex64 with
// each value rounded to the FP32 pair, within one ulp of (cos, sin) per
// component, whose modulus is closest to 1.  The forward and inverse passes
// use the same table (conjugated), so their phase roundings cancel and what
// repeats every step is the modulus error; choosing the pair this way cuts
// the complex64 drift per step by about 40 %.
int upload_tw(void** dst, const std::vector<cd>& v, int prec) {
    if (prec == SOFT_C128) return upload_c(dst, v, prec);
    std::vector<float> buf(2 * v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        const double c = v[i].real(), s = v[i].imag();
        const float c0 = (float)c, s0 = (float)s;
        float bc = c0, bs = s0;
        double be = 1e300, bd = 1e300;
        for (int dc = -1; dc <= 1; ++dc)
            for (int ds = -1; ds <= 1; ++ds) {
                const float cc = dc ? std::nextafter(c0, dc > 0 ? 2.0f : -2.0f) : c0;
                const float ss = ds ? std::nextafter(s0, ds > 0 ? 2.0f : -2.0f) : s0;
                const double e = std::fabs((double)cc * cc + (double)ss * ss - 1.0);
                const double d = std::fabs(cc - c) + std::fabs(ss - s);
                if (e < be || (e == be && d < bd)) { be = e; bd = d; bc = cc; bs = ss; }
            }
        buf[2 * i] = bc;
        buf[2 * i + 1] = bs;
    }
    return upload(dst, buf.data(), buf.size() * sizeof(float));
}

// Twiddle bases of the 1D step kernel: complex128 as is; complex64 as
// compensated float4 (hi.re, hi.im, lo.re, lo.im), hi + lo = the FP64 value
// to ~2^-48 (the kernel applies them by compensated multiplies, see
// soft1d.cuh)
int upload_tw_comp(void** dst, const std::vector<cd>& v, int prec) {
    return upload_tab(dst, v, prec);
}

// the upload_* conversions into a temporary device buffer, then one copy
// into dst
static int refill_with(int (*up)(void**, const std::vector<cd>&, int), void* dst,
                       const std::vector<cd>& v, int prec) {
    if (v.empty()) return SOFT_OK;
    const size_t bytes = v.size() * (prec == SOFT_C128 ? 16 : 8);
    void* tmp = nullptr;
    int rc = up(&tmp, v, prec);
    if (rc == SOFT_OK) rc = cuda_status(cudaMemcpy(dst, tmp, bytes, cudaMemcpyDeviceToDevice));
    cudaFree(tmp);
    return rc;
}
int refill_c(void* dst, const std::vector<cd>& v, int prec) { return refill_with(upload_c, dst, v, prec); }
int refill_vtab(void* dst, const std::vector<cd>& v, int prec) { return refill_with(upload_vtab, dst, v, prec); }

// Potential factors of one step from U0 (Sec. II, the scheme after Eq. C_FD):
// tv[j] = e^{-iU0 tau} off the strip block (both half factors merged),
// e^{-iU0 tau/2} on it (the strip CN sits between the halves); tvs holds
// the block rows' factors in the chunk layout of the strip CN (thread t of
// the n >> loge threads owns rows t*ch .. t*ch + ch - 1, entry c*T + t).
static void potential_tables_1d(const Tables1D& T, int n, double tau, std::vector<cd>& tv,
                                std::vector<cd>& tvs) {
    tv.resize(n);
    for (int j = 0; j < n; ++j) {
        const bool inblk = ((j - T.blk0 + n) % n) < T.nb;
        tv[j] = std::exp(cd(0.0, -1.0) * T.U0[j] * tau * (inblk ? 0.5 : 1.0));
    }
    tvs.clear();
    if (T.nb > 0) {
        const int thr = n >> T.loge, nb = T.nb;
        const int ch = (nb + thr - 1) / thr;
        tvs.assign((size_t)ch * thr, 1.0);
        for (int t = 0; t < thr; ++t)
            for (int c = 0; c < ch; ++c) {
                const int i = t * ch + c;
                if (i < nb) tvs[(size_t)c * thr + t] = tv[(T.blk0 + i) % n];
            }
    }
}

static int ilog2(int64_t n) {
    int l = 0;
    while ((int64_t(1) << l) < n) ++l;
    return (int64_t(1) << l) == n ? l : -1;
}

static void free_tables(Tables1D* t) {
    cudaFree(t->TK); cudaFree(t->TKh); cudaFree(t->TV); cudaFree(t->W); cudaFree(t->cn);
    cudaFree(t->TVs);
}

// Build (host FP64) and upload the tables of one 1D problem.
int make_tables_1d(Tables1D* T, int n, double a, double b, double R0, double theta, double tau,
                   const soft_options& o, int loge, int logrm) {
    const int logn = ilog2(n);
    T->prec = o.prec; T->logn = logn; T->loge = loge; T->logrm = logrm;
    T->R0 = R0; T->theta = theta;
    ContourFn cf(o.contour, R0, b, theta, o.tfecs_alpha, o.cap_energy, o.tfap_kmin);
    build_axis(T->ax, n, a, b, cf, tau);
    const Axis1D& A = T->ax;
    int rc = find_block(A, &T->blk0, &T->nb);
    if (rc) return rc;
    T->iL = 0; T->iR = 0;
    for (int j = 0; j < n; ++j) {
        if (A.x[j] <= -R0) T->iL = j + 1;
        if (A.x[j] < R0) T->iR = j + 1;
    }
    T->U0.resize(n);
    T->Uabs.resize(n);
    for (int j = 0; j < n; ++j) {
        T->Uabs[j] = cf.absorber(A.x[j]);
        T->U0[j] = soft_coulomb(&A.z[j], 1, o.soft_a2, o.charge) + T->Uabs[j];
    }
    // kinetic tables in the forward FFT's output order, 1/N folded in
    const std::vector<int> perm = dif_output_order(logn, logrm);
    std::vector<cd> tk(n), tkh(n), tv, tvs;
    const std::vector<cd> w = pass_twiddles(logn, logrm);
    // The step kernel reads them in its last forward pass, whose butterflies
    // hold R consecutive positions b*R + m (R its radix): entry (b, m) is
    // stored at m*(n/R) + b, so that a warp's reads are contiguous.
    const int lrl = (logn % logrm) ? logn % logrm : logrm;
    const int Rl = 1 << lrl, nbf = n >> lrl;
    for (int p = 0; p < n; ++p) {
        const double k = A.k[perm[p]];
        const int q = (p % Rl) * nbf + p / Rl;
        tk[q] = std::polar(1.0 / n, -0.5 * k * k * tau);
        tkh[q] = std::polar(1.0 / n, -0.25 * k * k * tau);
    }
    potential_tables_1d(*T, n, tau, tv, tvs);
    // Strip CN coefficients for the kernel's chunked solve: thread t of the
    // T = n >> loge threads owns rows t*ch .. t*ch + ch - 1 (ch = ceil(nb/T)).
    // M is complex symmetric, so mb_i = mf_{i+1}: the kernel reads mf of rows
    // t*ch + c, c <= ch, at c*T + t (0 past the block), then g of row t*ch + c
    // at (ch+1)*T + c*T + t (tvs holds the rows' potential factors).
    std::vector<cd> mf, mb, g, cnv;
    if (T->nb > 0) {
        double err = 0;
        rc = strip_factor(A, T->blk0, T->nb, mf, mb, g, &err);
        if (rc) return rc;
        const int thr = n >> loge, nb = T->nb;
        for (int i = 0; i + 1 < nb; ++i)
            if (std::abs(mb[i] - mf[i + 1]) > 1e-12 * (std::abs(mb[i]) + 1e-300)) return SOFT_ERR_SETUP;
        const int ch = (nb + thr - 1) / thr, P1 = (ch + 1) * thr;
        cnv.assign((size_t)P1 + (size_t)ch * thr, 0.0);
        for (int t = 0; t < thr; ++t)
            for (int c = 0; c <= ch; ++c) {
                const int i = t * ch + c;
                if (i < nb) cnv[(size_t)c * thr + t] = mf[i];
                if (c < ch && i < nb) cnv[P1 + (size_t)c * thr + t] = g[i];
            }
    }
    if ((rc = upload_tab(&T->TK, tk, o.prec))) return rc;
    if ((rc = upload_tab(&T->TKh, tkh, o.prec))) return rc;
    if ((rc = upload_vtab(&T->TV, tv, o.prec))) return rc;
    if (o.prec == SOFT_C128)   // every twiddle of the small-stride passes (see soft1d.cuh, TwFullD)
        rc = upload_c(&T->W, pass_twiddles_full(logn, logrm, TWFULL_MAXS), o.prec);
    else
        rc = upload_tw_comp(&T->W, w, o.prec);
    if (rc) return rc;
    if ((rc = upload_c(&T->cn, cnv, o.prec))) return rc;
    if ((rc = upload_vtab(&T->TVs, tvs, o.prec))) return rc;
    return SOFT_OK;
}

}  // namespace soft

// ------------------------------------------------------------------------ ABI
extern "C" {

void soft_default_options(soft_options* opt) {
    if (!opt) return;
    opt->prec = SOFT_C128;
    opt->contour = SOFT_CONTOUR_SHARP;
    opt->tfecs_alpha = 0.5;
    opt->soft_a2 = 2.0;
    opt->charge = 1.0;
    opt->band_width = 10;
    opt->autotune = 0;
    opt->cap_energy = 2.0;
    opt->tfap_kmin = 0.25;
    opt->persistent = 1;
}

const char* soft_strerror(int s) {
    switch (s) {
    case SOFT_OK: return "ok";
    case SOFT_ERR_INVALID_ARG: return "invalid argument";
    case SOFT_ERR_NOT_POW2: return "grid size must be a power of two in the supported range";
    case SOFT_ERR_OOM: return "device memory allocation failed";
    case SOFT_ERR_CUDA: return "CUDA runtime error";
    case SOFT_ERR_NOT_CONVERGED: return "PCG did not reach the tolerance within maxit";
    case SOFT_ERR_BREAKDOWN: return "PCG breakdown (vanishing bilinear form)";
    case SOFT_ERR_TIMEOUT: return "device wait timed out";
    case SOFT_ERR_NONFINITE: return "non-finite value in input or result";
    case SOFT_ERR_UNSUPPORTED: return "size/precision combination not supported";
    case SOFT_ERR_SETUP: return "plan tables failed a self-check";
    case SOFT_ERR_TOO_LARGE: return "request exceeds the fixed scratch of the no-allocation entry point";
    }
    return "unknown status";
}

static int check_opts(const soft_options* opt, soft_options* o) {
    soft_default_options(o);
    if (opt) *o = *opt;
    if (o->prec != SOFT_C64 && o->prec != SOFT_C128) return SOFT_ERR_INVALID_ARG;
    if (o->contour < 0 || o->contour > SOFT_ABSORB_TFAP) return SOFT_ERR_INVALID_ARG;
    if (!(o->cap_energy >= 0) || !(o->tfap_kmin >= 0) || !std::isfinite(o->cap_energy) ||
        !std::isfinite(o->tfap_kmin))
        return SOFT_ERR_INVALID_ARG;
    if (!(o->soft_a2 > 0) && o->charge != 0) return SOFT_ERR_INVALID_ARG;
    if (o->band_width < 1) return SOFT_ERR_INVALID_ARG;
    if (o->persistent != 0 && o->persistent != 1) return SOFT_ERR_INVALID_ARG;
    return SOFT_OK;
}

static int check_axis(int64_t n, double a, double b, double R0) {
    const int l = ilog2(n);
    if (l < 6 || l > 14) return SOFT_ERR_NOT_POW2;
    if (!(b > 0) || std::fabs(a + b) > 1e-12 * b) return SOFT_ERR_INVALID_ARG;
    if (!(R0 > 0 && R0 < b)) return SOFT_ERR_INVALID_ARG;
    return SOFT_OK;
}

// Time every built kernel variant of one 1D size on a sample of instances
// (up to four waves of the device's SMs) and return the fastest configuration.
static int autotune_size(const soft_options& o, int n, double a, double b, double R0, double theta,
                         double dt, int count, int* best_e, int* best_r) {
    int le[16], lr[16];
    const int logn = ilog2(n);
    const int nv = soft1d_variants(o.prec, logn, le, lr, 16);
    if (nv <= 1) return SOFT_OK;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        return SOFT_ERR_CUDA;
    const int ns = std::min(count, 4 * nsm);
    const size_t eb = o.prec == SOFT_C64 ? 8 : 16;
    void* psi = nullptr;
    int rc = cuda_status(cudaMalloc(&psi, eb * (size_t)ns * n));
    if (rc) return rc;
    cudaMemset(psi, 0x3c, eb * (size_t)ns * n);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int v = 0; v < nv && rc == SOFT_OK; ++v) {
        Tables1D T;
        if (make_tables_1d(&T, n, a, b, R0, theta, dt, o, le[v], lr[v]) == SOFT_OK) {
            const int thr = n >> le[v];
            if ((T.nb + thr - 1) / thr <= (1 << le[v]) / 4 + 2) {
                std::vector<Inst1D> d(ns);
                for (int i = 0; i < ns; ++i) {
                    std::memset(&d[i], 0, sizeof(Inst1D));
                    d[i].off = (int64_t)i * n;
                    d[i].TK = T.TK; d[i].TKh = T.TKh; d[i].TV = T.TV; d[i].W = T.W; d[i].cn = T.cn;
                    d[i].TVs = T.TVs;
                    d[i].nb = T.nb; d[i].blk0 = T.blk0; d[i].x0 = T.ax.x[0]; d[i].h = T.ax.h;
                    d[i].R0 = R0; d[i].tau = dt; d[i].iL = T.iL; d[i].iR = T.iR; d[i].n = n;
                }
                void* dd = nullptr;
                if (upload(&dd, d.data(), d.size() * sizeof(Inst1D)) == SOFT_OK) {
                    launch_soft1d(o.prec, logn, le[v], lr[v], (Inst1D*)dd, ns, psi, 2, nullptr, 0,
                                  nullptr, 0, nullptr);
                    cudaEventRecord(e0, 0);
                    launch_soft1d(o.prec, logn, le[v], lr[v], (Inst1D*)dd, ns, psi, 8, nullptr, 0,
                                  nullptr, 0, nullptr);
                    cudaEventRecord(e1, 0);
                    if (cudaEventSynchronize(e1) == cudaSuccess) {
                        float ms = 0;
                        cudaEventElapsedTime(&ms, e0, e1);
                        if (ms < best) { best = ms; *best_e = le[v]; *best_r = lr[v]; }
                    } else {
                        rc = SOFT_ERR_CUDA;
                    }
                }
                cudaFree(dd);
            }
        }
        free_tables(&T);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(psi);
    return rc;
}

// shared by soft_create (1D) and soft_create_batch
static int create_1d(int count, const soft_grid* grids, const double* boxes, const double* R0,
                     const double* theta, const soft_field* fields, double dt,
                     const soft_options& o, bool single, soft_plan** out) {
    std::unique_ptr<soft_plan> P(new soft_plan());
    P->kind = 1;
    P->single = single;
    P->prec = o.prec;
    P->opt = o;
    P->dt = dt;
    std::map<std::tuple<int64_t, double, double, double, double>, int> seen;
    std::map<std::pair<double, double>, int> cls;
    int64_t off = 0;
    for (int i = 0; i < count; ++i) {
        if (grids[i].ndim != 1) return SOFT_ERR_INVALID_ARG;
        const int64_t n = grids[i].n[0];
        const double a = boxes[2 * i], b = boxes[2 * i + 1];
        int rc = check_axis(n, a, b, R0[i]);
        if (rc) return rc;
        const int logn = ilog2(n);
        int loge, logrm, pgroups;
        soft1d_default_cfg(o.prec, logn, &loge, &logrm);
        // sizes of the persistent kernel keep its (elements per thread, radix)
        const bool persist = !single && o.persistent &&
                             persist_config(o.prec, logn, &loge, &logrm, &pgroups) >= 0;
        if (!persist && !soft1d_supported(o.prec, logn, loge, logrm)) return SOFT_ERR_UNSUPPORTED;
        auto key = std::make_tuple(n, a, b, R0[i], theta[i]);
        int tab;
        auto it = seen.find(key);
        if (it == seen.end()) {
            if (o.autotune && !persist) {
                int cnt = 0;
                for (int j = i; j < count; ++j)
                    if (grids[j].n[0] == n) ++cnt;
                rc = autotune_size(o, (int)n, a, b, R0[i], theta[i], dt, cnt, &loge, &logrm);
                if (rc) return rc;
            }
            std::unique_ptr<Tables1D> T(new Tables1D());
            rc = make_tables_1d(T.get(), (int)n, a, b, R0[i], theta[i], dt, o, loge, logrm);
            if (rc) { free_tables(T.get()); return rc; }
            // strip rows per thread must fit the kernel's register budget
            const int thr = (int)(n >> loge);
            const int chunk = (T->nb + thr - 1) / thr;
            if (chunk > (1 << loge) / 4 + 2) { free_tables(T.get()); return SOFT_ERR_UNSUPPORTED; }
            tab = (int)P->tabs.size();
            P->tabs.push_back(std::move(T));
            seen[key] = tab;
        } else {
            tab = it->second;
        }
        soft_plan::InstHost ih;
        ih.tab = tab; ih.off = off; ih.n = (int)n;
        ih.has_field = 0; ih.fcls = 0; ih.E0 = 0;
        if (fields) {
            const soft_field& f = fields[i];
            if (f.E0 != 0.0) {
                if (!(f.omega > 0 && f.ncycles > 0)) return SOFT_ERR_INVALID_ARG;
                const double Tp = f.ncycles * 2 * 3.14159265358979323846 / f.omega;
                auto k = std::make_pair(f.omega, Tp);
                auto c = cls.find(k);
                if (c == cls.end()) {
                    const int id = (int)P->h_cls.size() / 2;
                    P->h_cls.push_back(f.omega);
                    P->h_cls.push_back(Tp);
                    cls[k] = id;
                    ih.fcls = id;
                } else {
                    ih.fcls = c->second;
                }
                if (o.contour >= SOFT_ABSORB_CAP) return SOFT_ERR_UNSUPPORTED;   // absorbers: no field
                ih.has_field = 1;
                ih.E0 = f.E0;
            }
        }
        P->inst.push_back(ih);
        off += n;
    }
    P->total = off;
    int rc = P->build_1d_device();
    if (rc) return rc;
    if (!single && o.persistent && o.autotune && P->npacks > 0 && (rc = P->time_schedules())) return rc;
    *out = P.release();
    return SOFT_OK;
}

static int soft_create_impl(const soft_grid* grid, const double* box, double R0, double theta, double dt,
                            const soft_options* opt, soft_plan** out) {
    if (!grid || !box || !out) return SOFT_ERR_INVALID_ARG;
    *out = nullptr;
    if (!std::isfinite(dt) || dt == 0.0 || !std::isfinite(theta)) return SOFT_ERR_INVALID_ARG;
    soft_options o;
    int rc = check_opts(opt, &o);
    if (rc) return rc;
    if (grid->ndim == 1) return create_1d(1, grid, box, &R0, &theta, nullptr, dt, o, true, out);
    if (grid->ndim == 2) return create_2d(grid, box, R0, theta, dt, o, out);
    if (grid->ndim == 3) return create_3d(grid, box, R0, theta, dt, o, out);
    return SOFT_ERR_INVALID_ARG;
}
int soft_create(const soft_grid* grid, const double* box, double R0, double theta, double dt,
                const soft_options* opt, soft_plan** out) {
    return abi_guard([&] { return soft_create_impl(grid, box, R0, theta, dt, opt, out); });
}

static int soft_create_batch_impl(int count, const soft_grid* grids, const double* boxes, const double* R0,
                                  const double* theta, const soft_field* fields, double dt,
                                  const soft_options* opt, soft_plan** out) {
    if (count <= 0 || !grids || !boxes || !R0 || !theta || !out) return SOFT_ERR_INVALID_ARG;
    *out = nullptr;
    if (!std::isfinite(dt) || dt == 0.0) return SOFT_ERR_INVALID_ARG;
    soft_options o;
    int rc = check_opts(opt, &o);
    if (rc) return rc;
    return create_1d(count, grids, boxes, R0, theta, fields, dt, o, false, out);
}
int soft_create_batch(int count, const soft_grid* grids, const double* boxes, const double* R0,
                      const double* theta, const soft_field* fields, double dt,
                      const soft_options* opt, soft_plan** out) {
    return abi_guard([&] { return soft_create_batch_impl(count, grids, boxes, R0, theta, fields, dt, opt, out); });
}

int soft_batch_layout(const soft_plan* P, int64_t* offsets, int64_t* total) {
    if (!P || P->kind != 1) return SOFT_ERR_INVALID_ARG;
    if (offsets)
        for (size_t i = 0; i < P->inst.size(); ++i) offsets[i] = P->inst[i].off;
    if (total) *total = P->total;
    return SOFT_OK;
}

static int soft_step_impl(soft_plan* P, void* psi, int64_t nsteps, const soft_field* field, double* t_inout,
                          void* stream) {
    if (!P || !psi || !t_inout || nsteps < 0) return SOFT_ERR_INVALID_ARG;
    if (P->kind == 2) return P->step_2d(psi, nsteps, t_inout, (cudaStream_t)stream);
    if (P->kind == 3) return P->step_3d(psi, nsteps, t_inout, (cudaStream_t)stream);
    if (P->kind != 1) return SOFT_ERR_INVALID_ARG;
    if (P->single) {
        int rc = P->set_single_field(field, (cudaStream_t)stream);
        if (rc) return rc;
    }
    return P->step_1d(psi, nsteps, t_inout, (cudaStream_t)stream);
}
int soft_step(soft_plan* P, void* psi, int64_t nsteps, const soft_field* field, double* t_inout,
              void* stream) {
    return abi_guard([&] { return soft_step_impl(P, psi, nsteps, field, t_inout, stream); });
}

static int soft_step_batch_impl(soft_plan* P, void* psi, int64_t nsteps, double* t_inout, void* stream) {
    if (!P || !psi || !t_inout || nsteps < 0 || P->kind != 1) return SOFT_ERR_INVALID_ARG;
    return P->step_1d(psi, nsteps, t_inout, (cudaStream_t)stream);
}
int soft_step_batch(soft_plan* P, void* psi, int64_t nsteps, double* t_inout, void* stream) {
    return abi_guard([&] { return soft_step_batch_impl(P, psi, nsteps, t_inout, stream); });
}

int soft_observe(const soft_plan* P, const void* psi, double* norm_in, double* flux, void* stream) {
    if (!P || !psi || !norm_in || !flux || P->kind != 1) return SOFT_ERR_INVALID_ARG;
    int rc = launch_observe1d(P->prec, P->d_inst_obs, (int)P->inst.size(), psi, norm_in, flux,
                              (cudaStream_t)stream);
    const_cast<soft_plan*>(P)->last_launches = 1;
    return rc;
}

int soft_step_status(soft_plan* P, void* stream) {
    if (!P || P->kind != 1) return P ? SOFT_ERR_UNSUPPORTED : SOFT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    int rc = cuda_status(cudaMemcpyAsync(&h, P->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (rc == SOFT_OK) rc = cuda_status(cudaStreamSynchronize(st));
    if (rc) return rc;
    if (h == 0) return SOFT_OK;
    rc = cuda_status(cudaMemsetAsync(P->d_status, 0, sizeof(int), st));
    return rc ? rc : SOFT_ERR_NONFINITE;
}

static int soft_set_potential_impl(soft_plan* P, const double* U, int64_t n) {
    if (!P || !U || n <= 0) return SOFT_ERR_INVALID_ARG;
    for (int64_t i = 0; i < 2 * n; ++i)
        if (!std::isfinite(U[i])) return SOFT_ERR_NONFINITE;
    if (P->kind == 2) {
        if (n != (int64_t)P->p2->nx * P->p2->ny) return SOFT_ERR_INVALID_ARG;
        return P->p2->set_potential(U);
    }
    if (P->kind == 3) {
        if (n != P->points_3d()) return SOFT_ERR_INVALID_ARG;
        return P->p3->set_potential(U);
    }
    if (P->kind != 1 || !P->single || P->tabs.size() != 1) return SOFT_ERR_UNSUPPORTED;
    Tables1D* T = P->tabs[0].get();
    const int nn = 1 << T->logn;
    if (n != nn) return SOFT_ERR_INVALID_ARG;
    int rc = cuda_status(cudaDeviceSynchronize());      // no step may still read the tables
    if (rc) return rc;
    for (int j = 0; j < nn; ++j) T->U0[j] = cd(U[2 * j], U[2 * j + 1]) + T->Uabs[j];
    std::vector<cd> tv, tvs;
    potential_tables_1d(*T, nn, P->dt, tv, tvs);
    if ((rc = refill_vtab(T->TV, tv, T->prec))) return rc;
    if ((rc = refill_vtab(T->TVs, tvs, T->prec))) return rc;
    return sse1d_refill_potential(P);
}
int soft_set_potential(soft_plan* P, const double* U, int64_t n) {
    return abi_guard([&] { return soft_set_potential_impl(P, U, n); });
}

void soft_destroy(soft_plan* P) { delete P; }

int soft_plan_count(const soft_plan* P) {
    if (!P) return 0;
    return P->kind == 1 ? (int)P->inst.size() : 1;
}
int64_t soft_plan_points(const soft_plan* P, int i) {
    if (!P) return 0;
    if (P->kind == 1) return (i >= 0 && i < (int)P->inst.size()) ? P->inst[i].n : 0;
    return P->kind == 3 ? P->points_3d() : P->points_2d();
}
int soft_plan_prec(const soft_plan* P) { return P ? P->prec : 0; }
int64_t soft_last_launches(const soft_plan* P) { return P ? P->last_launches : 0; }

}  // extern "C"

// ---------------------------------------------------------------- soft_plan
soft_plan::~soft_plan() {
    for (auto& t : tabs) free_tables(t.get());
    for (auto& g : groups) cudaFree(g.d_inst);
    cudaFree(d_pinst);
    cudaFree(d_packs);
    cudaFree(d_pcount);
    cudaFree(d_inst_obs);
    cudaFree(d_cls);
    cudaFree(d_ftab);
    cudaFree(d_status);
    cudaFree(d_t0);
    delete nn;
    sse1d_free(s1);
    surf1d_free(sf);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (side_ready) {
        for (size_t g = 0; g < groups.size() && g < MAX_SIDE; ++g) {
            cudaStreamDestroy(side[g]);
            cudaEventDestroy(ev_join[g]);
        }
        cudaEventDestroy(ev_fork);
    }
    free_2d();
    free_3d();
}

Inst1D soft_plan::descriptor(int i) const {
    const InstHost& ih = inst[i];
    const Tables1D& T = *tabs[ih.tab];
    Inst1D d;
    std::memset(&d, 0, sizeof(d));
    d.off = ih.off;
    d.TK = T.TK; d.TKh = T.TKh; d.TV = T.TV; d.W = T.W; d.cn = T.cn; d.TVs = T.TVs;
    d.nb = T.nb; d.blk0 = T.blk0;
    d.x0 = T.ax.x[0]; d.h = T.ax.h; d.R0 = T.R0; d.tau = dt;
    d.E0 = ih.E0; d.has_field = ih.has_field; d.fcls = ih.fcls;
    d.iL = T.iL; d.iR = T.iR; d.n = ih.n;
    return d;
}

int soft_plan::build_1d_device() {
    // groups by kernel configuration, largest N first
    std::map<std::pair<int, int>, int> gid;
    for (size_t i = 0; i < inst.size(); ++i) {
        const Tables1D& T = *tabs[inst[i].tab];
        auto key = std::make_pair(-T.logn, T.loge * 8 + T.logrm);
        auto it = gid.find(key);
        if (it == gid.end()) {
            Group1D g;
            g.logn = T.logn; g.loge = T.loge; g.logrm = T.logrm;
            gid[key] = (int)groups.size();
            groups.push_back(g);
            it = gid.find(key);
        }
        groups[it->second].members.push_back((int)i);
    }
    std::sort(groups.begin(), groups.end(), [](const Group1D& a, const Group1D& b) { return a.logn > b.logn; });
    int rc;
    // the persistent kernel's sizes leave the group list: their instances
    // form packs of up to G same-size instances, largest N first
    if (!single && opt.persistent) {
        std::vector<Pack1D> packs;
        std::vector<Inst1D> pd;
        for (auto& g : groups) {
            int le, lr, G;
            const int v = persist_config(prec, g.logn, &le, &lr, &G);
            if (v < 0 || le != g.loge || lr != g.logrm) continue;
            g.in_persist = true;
            for (size_t k = 0; k < g.members.size(); k += G) {
                Pack1D pk;
                pk.var = v;
                pk.first = (int)pd.size();
                pk.count = (int)std::min<size_t>(G, g.members.size() - k);
                pk.pad_ = 0;
                for (int j = 0; j < pk.count; ++j) pd.push_back(descriptor(g.members[k + j]));
                packs.push_back(pk);
            }
        }
        std::stable_sort(packs.begin(), packs.end(), [](const Pack1D& a, const Pack1D& b) { return a.var < b.var; });
        npacks = (int)packs.size();
        use_persist = npacks > 0;
        if (npacks > 0) {
            if ((rc = upload((void**)&d_pinst, pd.data(), pd.size() * sizeof(Inst1D)))) return rc;
            if ((rc = upload(&d_packs, packs.data(), packs.size() * sizeof(Pack1D)))) return rc;
            if ((rc = cuda_status(cudaMalloc((void**)&d_pcount, sizeof(int))))) return rc;
            // sets the kernel's shared-memory attribute outside any capture
            if ((rc = launch_persist(prec, nullptr, 0, nullptr, nullptr, nullptr, 0, nullptr, 0, nullptr, 0,
                                     nullptr)))
                return rc;
        }
    }
    for (auto& g : groups) {
        std::vector<Inst1D> d;
        for (int i : g.members) d.push_back(descriptor(i));
        if ((rc = upload((void**)&g.d_inst, d.data(), d.size() * sizeof(Inst1D)))) return rc;
    }
    h_obs.clear();
    for (size_t i = 0; i < inst.size(); ++i) h_obs.push_back(descriptor((int)i));
    if ((rc = upload((void**)&d_inst_obs, h_obs.data(), h_obs.size() * sizeof(Inst1D)))) return rc;
    ncls = (int)h_cls.size() / 2;
    // room for one extra class used by soft_step's per-call field
    std::vector<double> c = h_cls;
    c.push_back(1.0); c.push_back(1.0);
    if ((rc = upload((void**)&d_cls, c.data(), c.size() * sizeof(double)))) return rc;
    ftab_cap = 4096;
    if ((rc = cuda_status(cudaMalloc((void**)&d_ftab, sizeof(double) * ftab_cap * (ncls + 1))))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&d_status, sizeof(int))))) return rc;
    if ((rc = cuda_status(cudaMemset(d_status, 0, sizeof(int))))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&d_t0, sizeof(double))))) return rc;
    return SOFT_OK;
}

// soft_step on a single-instance plan: the call's field replaces the plan's.
// The descriptor and pulse-class copies are queued on the call's stream, so
// they take effect after every step already queued there (a step still
// waiting on a non-blocking stream keeps the field it was called with);
// pageable sources are staged before cudaMemcpyAsync returns.
int soft_plan::set_single_field(const soft_field* f, cudaStream_t st) {
    InstHost& ih = inst[0];
    int has = 0, fc = 0;
    double E0 = 0;
    if (f && f->E0 != 0.0) {
        if (!(f->omega > 0 && f->ncycles > 0)) return SOFT_ERR_INVALID_ARG;
        if (opt.contour >= SOFT_ABSORB_CAP) return SOFT_ERR_UNSUPPORTED;   // absorbers: no field
        const double Tp = f->ncycles * 2 * 3.14159265358979323846 / f->omega;
        if (call_cls[0] != f->omega || call_cls[1] != Tp) {
            call_cls[0] = f->omega;
            call_cls[1] = Tp;
            int rc = cuda_status(cudaMemcpyAsync(d_cls + 2 * ncls, call_cls, 2 * sizeof(double),
                                                 cudaMemcpyHostToDevice, st));
            if (rc) return rc;
        }
        has = 1; fc = ncls; E0 = f->E0;
    }
    if (has != ih.has_field || fc != ih.fcls || E0 != ih.E0) {
        ih.has_field = has; ih.fcls = fc; ih.E0 = E0;
        Inst1D d = descriptor(0);
        for (auto& g : groups) {
            int rc = cuda_status(cudaMemcpyAsync(g.d_inst, &d, sizeof(d), cudaMemcpyHostToDevice, st));
            if (rc) return rc;
        }
        h_obs[0] = d;
        int rc = cuda_status(cudaMemcpyAsync(d_inst_obs, &d, sizeof(d), cudaMemcpyHostToDevice, st));
        if (rc) return rc;
    }
    return SOFT_OK;
}

// one chunk of steps on the given stream: pulse table from the device start
// time, the persistent kernel (if used) and the size groups on parallel
// branches, then the start time advanced
int soft_plan::enqueue_chunk(void* psi, int64_t chunk, cudaStream_t st) {
    const int nc = ncls + (single ? 1 : 0);
    int rc;
    if (nc > 0) {
        if ((rc = launch_field_table_dev(d_cls, nc, d_t0, dt, chunk, d_ftab, ftab_cap, st))) return rc;
        ++last_launches;
    }
    const bool persist = use_persist && npacks > 0;
    int nlaunch = persist ? 1 : 0;
    for (const auto& G : groups)
        if (!(persist && G.in_persist)) ++nlaunch;
    const bool fork = nlaunch > 1;
    if (fork && (rc = cuda_status(cudaEventRecord(ev_fork, st)))) return rc;
    if (persist) {           // the persistent kernel on the call's stream, the groups beside it
        if ((rc = cuda_status(cudaMemsetAsync(d_pcount, 0, sizeof(int), st)))) return rc;
        if ((rc = launch_persist(prec, d_packs, npacks, d_pcount, d_pinst, psi, chunk, d_ftab, ftab_cap, d_status,
                                 st, nullptr)))
            return rc;
        last_launches += 1;
    }
    for (size_t g = 0; g < groups.size(); ++g) {
        if (persist && groups[g].in_persist) continue;
        cudaStream_t gs = fork ? side[g] : st;
        if (fork && (rc = cuda_status(cudaStreamWaitEvent(gs, ev_fork, 0)))) return rc;
        const Group1D& G = groups[g];
        rc = launch_soft1d(prec, G.logn, G.loge, G.logrm, G.d_inst, (int)G.members.size(), psi, chunk,
                           d_ftab, ftab_cap, d_status, gs, nullptr);
        if (rc) return rc;
        ++last_launches;
        if (fork) {
            if ((rc = cuda_status(cudaEventRecord(ev_join[g], gs)))) return rc;
            if ((rc = cuda_status(cudaStreamWaitEvent(st, ev_join[g], 0)))) return rc;
        }
    }
    if ((rc = launch_advance_time(d_t0, (double)chunk * dt, st))) return rc;
    ++last_launches;
    return SOFT_OK;
}

int soft_plan::ensure_side() {
    int rc;
    if (!side_ready) {
        for (size_t g = 0; g < groups.size() && g < MAX_SIDE; ++g) {
            if ((rc = cuda_status(cudaStreamCreateWithFlags(&side[g], cudaStreamNonBlocking)))) return rc;
            if ((rc = cuda_status(cudaEventCreateWithFlags(&ev_join[g], cudaEventDisableTiming)))) return rc;
        }
        if ((rc = cuda_status(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming)))) return rc;
        side_ready = true;
    }
    return groups.size() > MAX_SIDE ? SOFT_ERR_UNSUPPORTED : SOFT_OK;
}

// The schedule autotuner of a batch plan: one chunk of 16 steps on a zero
// state with the persistent kernel and with one kernel per size group
// (each timed after a warm-up run); the faster is kept.
int soft_plan::time_schedules() {
    int rc = ensure_side();
    if (rc) return rc;
    const size_t eb = prec == SOFT_C64 ? 8 : 16;
    void* tmp = nullptr;
    if ((rc = cuda_status(cudaMalloc(&tmp, eb * (size_t)total)))) return rc;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms[2] = {0, 0};
    rc = cuda_status(cudaMemset(tmp, 0, eb * (size_t)total));
    if (!rc) rc = cuda_status(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    if (!rc) rc = cuda_status(cudaEventCreate(&e0));
    if (!rc) rc = cuda_status(cudaEventCreate(&e1));
    for (int mode = 0; mode < 2 && !rc; ++mode) {
        use_persist = mode == 0;
        const double zero = 0.0;
        rc = cuda_status(cudaMemcpyAsync(d_t0, &zero, sizeof(double), cudaMemcpyHostToDevice, st));
        for (int rep = 0; rep < 2 && !rc; ++rep) {
            if (rep == 1) rc = cuda_status(cudaEventRecord(e0, st));
            if (!rc) rc = enqueue_chunk(tmp, 16, st);
            if (!rc && rep == 1) rc = cuda_status(cudaEventRecord(e1, st));
        }
        if (!rc) rc = cuda_status(cudaEventSynchronize(e1));
        if (!rc) rc = cuda_status(cudaEventElapsedTime(&ms[mode], e0, e1));
    }
    use_persist = rc == SOFT_OK && ms[0] <= ms[1];
    last_launches = 0;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(tmp);
    return rc;
}

int soft_plan::step_1d(void* psi, int64_t nsteps, double* t_inout, cudaStream_t st) {
    last_launches = 0;
    if (nsteps == 0) return SOFT_OK;
    int rc;
    if ((rc = ensure_side())) return rc;
    // start time: a pageable copy is consumed before the call returns
    const double t0 = *t_inout;
    if ((rc = cuda_status(cudaMemcpyAsync(d_t0, &t0, sizeof(double), cudaMemcpyHostToDevice, st)))) return rc;
    int64_t done = 0;
    while (done < nsteps) {
        const int64_t chunk = std::min<int64_t>(ftab_cap, nsteps - done);
        if (!gexec || gpsi != psi || gchunk != chunk || gstream != st) {
            if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
            cudaStream_t cap;
            if ((rc = cuda_status(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)))) return rc;
            cudaGraph_t graph;
            const int64_t before = last_launches;
            rc = cuda_status(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
            if (rc == SOFT_OK) rc = enqueue_chunk(psi, chunk, cap);
            cudaError_t e = cudaStreamEndCapture(cap, &graph);
            if (rc == SOFT_OK) rc = cuda_status(e);
            if (rc == SOFT_OK) rc = cuda_status(cudaGraphInstantiate(&gexec, graph, 0));
            if (e == cudaSuccess) cudaGraphDestroy(graph);
            cudaStreamDestroy(cap);
            if (rc) { gexec = nullptr; return rc; }
            glaunches = last_launches - before;
            last_launches = before;
            gpsi = psi; gchunk = chunk; gstream = st;
        }
        if ((rc = cuda_status(cudaGraphLaunch(gexec, st)))) return rc;
        last_launches += glaunches;
        done += chunk;
    }
    *t_inout = t0 + (double)nsteps * dt;
    return SOFT_OK;
}
