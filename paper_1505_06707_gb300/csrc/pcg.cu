// Stationary ECS equation (Sec. III): host driver of the batched
// complex-symmetric CG with the FFT preconditioners, and the single
// applications of A and P^-1.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "band.h"
#include "nn.h"
#include "pcg.cuh"
#include "pcg_launch.h"
#include "plan_internal.h"

using namespace soft;

namespace soft {

struct PcgTables {               // one preconditioner type
    PcgGeo geo{};
    void* bufs[20] = {nullptr};
    int nb = 0;
};

struct Pcg {
    int nEcap = 0;
    int64_t N = 0;
    void *r = nullptr, *z = nullptr, *p = nullptr, *w = nullptr, *t = nullptr;
    double* dE = nullptr;
    double2* part = nullptr;
    double2* part2 = nullptr;
    int nparts_max = 0;
    // per-energy state (device)
    double2 *rho = nullptr, *alpha = nullptr, *beta = nullptr;
    double *relres = nullptr, *fnorm2 = nullptr;
    int *active = nullptr, *iters = nullptr, *status = nullptr, *nactive = nullptr;
    double* rref = nullptr;      // reliable updates of the FP32-A iteration
    int *upd = nullptr, *lastu = nullptr, *mode = nullptr, *act32 = nullptr, *act64 = nullptr;
    // A tables in FP64 and FP32, and the preconditioners
    void *U = nullptr, *Cx = nullptr, *Cy = nullptr, *Kx = nullptr, *Ky = nullptr;
    void *U32 = nullptr, *Cx32 = nullptr, *Cy32 = nullptr, *Kx32 = nullptr, *Ky32 = nullptr;
    PcgTables pc[3];             // simple, banded, banded with FP32 tables (and the FP32 A)
    bool tables = false;
    // flexible GCR: GCR_M stored direction pairs per energy
    static constexpr int GCR_M = 16;
    void *gP = nullptr, *gQ = nullptr;
    double2 *gbeta = nullptr, *gpart = nullptr;
    double* gqn = nullptr;
    int gcap = 0;
    ~Pcg() {
        void* v[] = {r, z, p, w, t, dE, part, part2, rho, alpha, beta, relres, fnorm2, active, iters,
                     status, nactive, rref, upd, lastu, mode, act32, act64, U, Cx, Cy, Kx, Ky, U32, Cx32, Cy32, Kx32, Ky32,
                     gP, gQ, gbeta, gpart, gqn};
        for (void* b : v) cudaFree(b);
        for (auto& T : pc)
            for (void* b : T.bufs) cudaFree(b);
    }
};

static int upload_i(void** dst, const std::vector<int>& v) {
    return upload(dst, v.data(), v.size() * sizeof(int));
}

// k^2/(2n) in the FFT output order of the given pass structure (real, phase-table format)
static std::vector<cd> ksq_tab(const Axis1D& A, int logn, int logrm) {
    const std::vector<int> perm = dif_output_order(logn, logrm);
    std::vector<cd> t(A.n);
    for (int p = 0; p < A.n; ++p) {
        const double k = A.k[perm[p]];
        t[p] = 0.5 * k * k / A.n;
    }
    return t;
}

static int build_pc(Plan2D* Q, int type, PcgTables& T, int prec = SOFT_C128) {
    const bool simple = type == 0;
    BandAxis bx, by;
    double chk;
    const int nbw = Q->band_width;
    int rc;
    if ((rc = build_band_axis(Q->ax, nbw, simple, bx, &chk))) return rc;
    if ((rc = build_band_axis(Q->ay, nbw, simple, by, &chk))) return rc;
    auto inv_perm = [](int logn, int logrm) {
        const std::vector<int> perm = dif_output_order(logn, logrm);
        std::vector<int> pos(perm.size());
        for (size_t p = 0; p < perm.size(); ++p) pos[perm[p]] = (int)p;
        return pos;
    };
    int i = 0;
    auto ub = [&](const std::vector<int>& v) -> const int* {
        void* d = nullptr;
        if (upload_i(&d, v)) return nullptr;
        T.bufs[i++] = d;
        return (const int*)d;
    };
    auto uc = [&](const std::vector<cd>& v) -> const void* {
        void* d = nullptr;
        if (upload_c(&d, v, prec)) return nullptr;
        T.bufs[i++] = d;
        return d;
    };
    PcgGeo& g = T.geo;
    g.posx = ub(inv_perm(Q->lx, Q->lrx));
    g.posy = ub(inv_perm(Q->ly, Q->lry));
    g.bsx = ub(bx.start); g.bsy = ub(by.start);
    g.bwx = ub(bx.width); g.bwy = ub(by.width);
    // band rows u-major (entry u of row nu at u * n + nu), zero past each width
    auto umajor = [](const BandAxis& B, const std::vector<cd>& tab) {
        int wmax = 0;
        for (int wd : B.width) wmax = std::max(wmax, wd);
        std::vector<cd> t((size_t)wmax * B.n, cd(0.0, 0.0));
        for (int nu = 0; nu < B.n; ++nu)
            for (int u = 0; u < B.width[nu]; ++u) t[(size_t)u * B.n + nu] = tab[(size_t)B.off[nu] + u];
        return t;
    };
    g.xfx = uc(umajor(bx, bx.xf)); g.xfy = uc(umajor(by, by.xf));
    g.xbx = uc(umajor(bx, bx.xb)); g.xby = uc(umajor(by, by.xb));
    g.lamx = uc(bx.lam); g.lamy = uc(by.lam);
    {                            // FFT twiddles (the four bases per pass)
        auto ut = [&](const std::vector<cd>& v) -> const void* {
            void* d = nullptr;
            if (upload_tw(&d, v, prec)) return nullptr;
            T.bufs[i++] = d;
            return d;
        };
        g.Wx = ut(pass_twiddles(Q->lx, Q->lrx));
        g.Wy = ut(pass_twiddles(Q->ly, Q->lry));
    }
    for (int k = 0; k < i; ++k)
        if (!T.bufs[k]) return SOFT_ERR_OOM;
    T.nb = i;
    return SOFT_OK;
}

static int ensure_tables(Plan2D* Q) {
    if (!Q->pcg) Q->pcg = new Pcg();
    Pcg* S = Q->pcg;
    if (S->tables) return SOFT_OK;
    S->N = (int64_t)Q->nx * Q->ny;
    int rc;
    if ((rc = upload_c(&S->U, Q->U, SOFT_C128))) return rc;
    auto cat = [](const Axis1D& A) {
        std::vector<cd> v = A.Cs;
        v.insert(v.end(), A.Cd.begin(), A.Cd.end());
        v.insert(v.end(), A.Cu.begin(), A.Cu.end());
        return v;
    };
    if ((rc = upload_c(&S->Cx, cat(Q->ax), SOFT_C128))) return rc;
    if ((rc = upload_c(&S->Cy, cat(Q->ay), SOFT_C128))) return rc;
    if ((rc = upload_tab(&S->Kx, ksq_tab(Q->ax, Q->lx, Q->lrx), SOFT_C128))) return rc;
    if ((rc = upload_tab(&S->Ky, ksq_tab(Q->ay, Q->ly, Q->lry), SOFT_C128))) return rc;
    if ((rc = upload_c(&S->U32, Q->U, SOFT_C64))) return rc;
    if ((rc = upload_c(&S->Cx32, cat(Q->ax), SOFT_C64))) return rc;
    if ((rc = upload_c(&S->Cy32, cat(Q->ay), SOFT_C64))) return rc;
    if ((rc = upload_tab(&S->Kx32, ksq_tab(Q->ax, Q->lx, Q->lrx), SOFT_C64))) return rc;
    if ((rc = upload_tab(&S->Ky32, ksq_tab(Q->ay, Q->ly, Q->lry), SOFT_C64))) return rc;
    for (int type = 0; type < 3; ++type) {
        const bool f32 = type == 2;
        if ((rc = build_pc(Q, f32 ? 1 : type, S->pc[type], f32 ? SOFT_C64 : SOFT_C128))) return rc;
        PcgGeo& g = S->pc[type].geo;
        g.nx = Q->nx; g.ny = Q->ny; g.N = S->N;
        g.Kx = f32 ? S->Kx32 : S->Kx; g.Ky = f32 ? S->Ky32 : S->Ky; g.U = f32 ? S->U32 : S->U;
        g.Cx = f32 ? S->Cx32 : S->Cx; g.Cy = f32 ? S->Cy32 : S->Cy;
        g.nbx = Q->geo.nbx; g.blk0x = Q->geo.blk0x; g.nby = Q->geo.nby; g.blk0y = Q->geo.blk0y;
    }
    // set the kernels' shared-memory attributes outside any capture
    for (int which = 0; which < 3; ++which)
        if ((rc = pcg_row(Q->lx, which, S->pc[0].geo, nullptr, nullptr, nullptr, nullptr, nullptr,
                          nullptr, 0, 0)))
            return rc;
    for (int which = 0; which < 2; ++which)
        if ((rc = pcg_col(Q->ly, which, S->pc[0].geo, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0)))
            return rc;
    for (int which = 1; which < 3; ++which)
        if ((rc = pcg_pc32_row(Q->lx, which, S->pc[2].geo, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0)))
            return rc;
    if ((rc = pcg_pc32_col(Q->ly, S->pc[2].geo, nullptr, nullptr, nullptr, 0, 0))) return rc;
    if ((rc = pcg_a32_row(Q->lx, S->pc[2].geo, nullptr, nullptr, nullptr, nullptr, 0, 0))) return rc;
    if ((rc = pcg_a32_col(Q->ly, S->pc[2].geo, nullptr, nullptr, nullptr, nullptr, 0, 0, 0))) return rc;
    S->tables = true;
    return SOFT_OK;
}

static int ensure_workspace(Plan2D* Q, int nE) {
    int rc = ensure_tables(Q);
    if (rc) return rc;
    Pcg* S = Q->pcg;
    if (S->nEcap >= nE) return SOFT_OK;
    void* v[] = {S->r, S->z, S->p, S->w, S->t, S->dE, S->part, S->part2, S->rho, S->alpha, S->beta,
                 S->relres, S->active, S->iters, S->status, S->rref, S->upd, S->lastu, S->mode,
                 S->act32, S->act64};
    for (void* b : v) cudaFree(b);
    S->r = S->z = S->p = S->w = S->t = nullptr;
    S->dE = S->relres = S->rref = nullptr;
    S->part = S->part2 = S->rho = S->alpha = S->beta = nullptr;
    S->active = S->iters = S->status = S->upd = S->lastu = S->mode = S->act32 = S->act64 = nullptr;
    S->nEcap = 0;
    const size_t vb = sizeof(double2) * (size_t)S->N * nE;
    S->nparts_max = std::max(std::max(Q->ny, pcg_col_blocks(Q->nx)), 256);
    if ((rc = cuda_status(cudaMalloc(&S->r, vb)))) return rc;
    if ((rc = cuda_status(cudaMalloc(&S->z, vb)))) return rc;
    if ((rc = cuda_status(cudaMalloc(&S->p, vb)))) return rc;
    if ((rc = cuda_status(cudaMalloc(&S->w, vb)))) return rc;
    if ((rc = cuda_status(cudaMalloc(&S->t, vb)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->dE, sizeof(double) * nE)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->part, sizeof(double2) * (size_t)nE * S->nparts_max)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->part2, sizeof(double2) * (size_t)nE * S->nparts_max)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->rho, sizeof(double2) * nE)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->alpha, sizeof(double2) * nE)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->beta, sizeof(double2) * nE)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->relres, sizeof(double) * nE)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->active, sizeof(int) * nE)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->iters, sizeof(int) * nE)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->status, sizeof(int) * nE)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->rref, sizeof(double) * nE)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->upd, sizeof(int) * nE)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->lastu, sizeof(int) * nE)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->mode, sizeof(int) * nE)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->act32, sizeof(int) * nE)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->act64, sizeof(int) * nE)))) return rc;
    if (!S->fnorm2 && (rc = cuda_status(cudaMalloc((void**)&S->fnorm2, sizeof(double))))) return rc;
    if (!S->nactive && (rc = cuda_status(cudaMalloc((void**)&S->nactive, sizeof(int))))) return rc;
    S->nEcap = nE;
    return SOFT_OK;
}

// z = P^-1 r for nE energies; with part, the per-row partials of r^T z
// type: 0 simple, 1 banded, 4 banded computing in FP32 (r, z complex128)
static int apply_pc(Plan2D* Q, int type, const void* r, void* z, const double* dE, const int* act,
                    double2* part, int nE, cudaStream_t st) {
    Pcg* S = Q->pcg;
    int rc;
    if (type == 4) {
        const PcgGeo& g = S->pc[2].geo;
        if ((rc = pcg_pc32_row(Q->lx, 1, g, r, S->t, nullptr, act, nullptr, nE, st))) return rc;
        if ((rc = pcg_pc32_col(Q->ly, g, S->t, dE, act, nE, st))) return rc;
        Q->launches += 3;
        return pcg_pc32_row(Q->lx, 2, g, S->t, z, part ? r : nullptr, act, part, nE, st);
    }
    const PcgGeo& g = S->pc[type].geo;
    if ((rc = pcg_row(Q->lx, 1, g, r, S->t, nullptr, dE, act, nullptr, nE, st))) return rc;
    if ((rc = pcg_col(Q->ly, 1, g, nullptr, S->t, dE, act, nullptr, nE, st))) return rc;
    Q->launches += 3;
    return pcg_row(Q->lx, 2, g, S->t, z, part ? r : nullptr, dE, act, part, nE, st);
}

// w = A p; with part, the per-column-block partials of p^T w
static int apply_A(Plan2D* Q, const void* p, void* w, const double* dE, const int* act,
                   double2* part, int nE, cudaStream_t st) {
    Pcg* S = Q->pcg;
    const PcgGeo& g = S->pc[0].geo;
    int rc;
    if ((rc = pcg_row(Q->lx, 0, g, p, w, nullptr, dE, act, nullptr, nE, st))) return rc;
    Q->launches += 2;
    return pcg_col(Q->ly, 0, g, p, w, dE, act, part, nE, st);
}

// ||f - A x_e|| / ||f|| in FP64 for the energies with act[e] (the device
// active flags must equal act); r holds the residuals afterwards
static int true_relres(Plan2D* Q, const void* rhs, const void* x, int nE, const std::vector<int>& act,
                       std::vector<double>& rel, cudaStream_t st) {
    Pcg* S = Q->pcg;
    const int64_t N = S->N;
    const int np = 256;
    int rc;
    if ((rc = apply_A(Q, x, S->w, S->dE, S->active, S->part2, nE, st))) return rc;
    if ((rc = vec_sub(rhs, S->w, S->r, S->active, N, nE, st))) return rc;
    if ((rc = vec_norm2(rhs, N, S->part2, np, st))) return rc;
    for (int e = 0; e < nE; ++e)
        if (act[e] && (rc = vec_norm2(static_cast<const double2*>(S->r) + (int64_t)e * N, N,
                                      S->part + (int64_t)e * np, np, st)))
            return rc;
    Q->launches += 3 + nE;
    std::vector<double2> pf(np), pr((size_t)nE * np);
    if ((rc = cuda_status(cudaMemcpyAsync(pf.data(), S->part2, sizeof(double2) * np, cudaMemcpyDeviceToHost, st)))) return rc;
    if ((rc = cuda_status(cudaMemcpyAsync(pr.data(), S->part, sizeof(double2) * pr.size(), cudaMemcpyDeviceToHost, st)))) return rc;
    if ((rc = cuda_status(cudaStreamSynchronize(st)))) return rc;
    double f2 = 0.0;
    for (const double2& v : pf) f2 += v.x;
    for (int e = 0; e < nE; ++e) {
        if (!act[e]) continue;
        double r2 = 0.0;
        for (int i = 0; i < np; ++i) r2 += pr[(size_t)e * np + i].x;
        rel[e] = std::sqrt(r2 / f2);
    }
    return SOFT_OK;
}

// COCG (Sec. III) with preconditioner type precond (0, 1 or 4) over the
// energies in s.active, from x = 0 or (warm) from the x already in psi_out
static int solve_cocg(Plan2D* Q, const PcgState& s, const void* rhs, void* psi_out, int maxit, int nE,
                      int precond, bool warm, cudaStream_t st) {
    Pcg* S = Q->pcg;
    const int64_t N = S->N;
    const int np_row = Q->ny, np_vec = 256, np_col = pcg_col_blocks(Q->nx);
    int rc;
    if (warm) {                              // r = f - A x for the active energies
        if ((rc = apply_A(Q, psi_out, S->w, S->dE, S->active, S->part2, nE, st))) return rc;
        if ((rc = vec_sub(rhs, S->w, S->r, S->active, N, nE, st))) return rc;
        Q->launches += 1;
    } else if ((rc = vec_init(rhs, psi_out, S->r, N, nE, st))) {     // x = 0, r = f
        return rc;
    }
    // ||f||^2, z = P^-1 r, rho = r^T z, p = z
    if ((rc = vec_norm2(rhs, N, S->part, np_vec, st))) return rc;
    if ((rc = pcg_scalars(STAGE_FNORM, nE, S->part, np_vec, s, st))) return rc;
    // COCG (Sec. III): z = P^-1 r, rho = r^T z, p = z
    if ((rc = apply_pc(Q, precond, S->r, S->z, S->dE, S->active, S->part, nE, st))) return rc;
    if ((rc = pcg_scalars(STAGE_RHO, nE, S->part, np_row, s, st))) return rc;
    if ((rc = vec_p(S->p, S->z, S->beta, S->active, N, nE, 1, st))) return rc;
    Q->launches += 5;
    const int CHECK = 4;
    for (int it = 1; it <= maxit; ++it) {
        if ((rc = apply_A(Q, S->p, S->w, S->dE, S->active, S->part, nE, st))) return rc;
        if ((rc = pcg_scalars(STAGE_ALPHA, nE, S->part, np_col, s, st))) return rc;
        if ((rc = vec_xr(psi_out, S->r, S->p, S->w, S->alpha, S->active, N, nE, S->part, np_vec, st))) return rc;
        if ((rc = pcg_scalars(STAGE_RNORM, nE, S->part, np_vec, s, st))) return rc;
        Q->launches += 3;
        if (it % CHECK == 0 || it == maxit) {
            int na = 0;
            if ((rc = cuda_status(cudaMemcpyAsync(&na, S->nactive, sizeof(int), cudaMemcpyDeviceToHost, st)))) return rc;
            if ((rc = cuda_status(cudaStreamSynchronize(st)))) return rc;
            if (na <= 0) break;
        }
        if (it == maxit) break;
        if (precond == 4) {
            // FP32 preconditioner: not exactly symmetric, so the flexible
            // beta = z'^T (r' - r) / rho = -alpha z'^T w / rho
            if ((rc = apply_pc(Q, precond, S->r, S->z, S->dE, S->active, nullptr, nE, st))) return rc;
            if ((rc = vec_dot2(S->r, S->z, S->w, S->active, N, nE, S->part, S->part2, np_vec, st))) return rc;
            if ((rc = pcg_scalars(STAGE_BETA_FLEX, nE, S->part, np_vec, s, st, S->part2))) return rc;
            Q->launches += 1;
        } else {
            if ((rc = apply_pc(Q, precond, S->r, S->z, S->dE, S->active, S->part, nE, st))) return rc;
            if ((rc = pcg_scalars(STAGE_BETA, nE, S->part, np_row, s, st))) return rc;
        }
        if ((rc = vec_p(S->p, S->z, S->beta, S->active, N, nE, 0, st))) return rc;
        Q->launches += 5;
    }
    return SOFT_OK;
}

// w = A p on complex64 vectors (mixed iteration): A computing in FP32 for
// the energies in act32 (all if null), in FP64 for those in act64 (none if
// null); partials of p^T w at the stride of the FP64 column pass
static int apply_A_mixed(Plan2D* Q, const void* p, void* w, const double* dE, const int* act32,
                         const int* act64, double2* part, int nE, cudaStream_t st) {
    Pcg* S = Q->pcg;
    const int ps = pcg_col_blocks(Q->nx);
    int rc;
    if ((rc = pcg_a32_row(Q->lx, S->pc[2].geo, p, w, dE, act32, nE, st))) return rc;
    if ((rc = pcg_a32_col(Q->ly, S->pc[2].geo, p, w, act32, part, ps, nE, st))) return rc;
    Q->launches += 2;
    if (!act64) return SOFT_OK;
    if ((rc = pcg_a64f_row(Q->lx, S->pc[0].geo, p, w, dE, act64, nE, st))) return rc;
    Q->launches += 2;
    return pcg_a64f_col(Q->ly, S->pc[0].geo, p, w, act64, part, ps, nE, st);
}

// z = P^-1 r, banded preconditioner in FP32 on complex64 vectors; with part
// the per-row partials of r^T z, with w also those of z^T w in part2
static int apply_pc_mixed(Plan2D* Q, const void* r, void* z, const void* w, const double* dE,
                          const int* act, double2* part, double2* part2, int nE, cudaStream_t st) {
    Pcg* S = Q->pcg;
    const PcgGeo& g = S->pc[2].geo;
    int rc;
    if ((rc = pcg_pc32f_row(Q->lx, 1, g, r, S->t, nullptr, nullptr, act, nullptr, nullptr, nE, st))) return rc;
    if ((rc = pcg_pc32_col(Q->ly, g, S->t, dE, act, nE, st))) return rc;
    Q->launches += 3;
    return pcg_pc32f_row(Q->lx, 2, g, S->t, z, part ? r : nullptr, w, act, part, part2, nE, st);
}

// The mixed iteration (precond 5): COCG with the flexible beta in which A
// and the banded preconditioner compute in FP32 on complex64 r, p, z, w, and
// the solution increment since the last update accumulates in double-float.
// Reliable updates: once an energy's recursive residual has dropped by delta
// (or below tol, or maxgap iterations passed) the increment is folded into
// the complex128 x and the residual replaced by f - A x with A in FP64; only
// that true residual decides convergence.  An energy whose true residual has
// not halved since its previous update switches to the FP64 A (on the same
// complex64 vectors) after a restart; if it stalls again it leaves with mode
// bit 2 set, and the caller restarts it in FP64 (solve_cocg, warm).
static int solve_mixed(Plan2D* Q, const PcgState& s, const void* rhs, void* psi_out, int maxit, int nE,
                       cudaStream_t st) {
    Pcg* S = Q->pcg;
    const int64_t N = S->N, NE = N * nE;
    float2* r = (float2*)S->r;             // each complex128 buffer holds two complex64 vectors
    float2* xh = r + NE;
    float2* z = (float2*)S->z;
    float2* xl = z + NE;
    float2* p = (float2*)S->p;
    float2* w = (float2*)S->w;
    const int np_row = Q->ny, np_vec = 256, np_col = pcg_col_blocks(Q->nx);
    int rc;
    // x = 0, r = f, ||f||^2, z = P^-1 r, rho = r^T z, p = z
    if ((rc = vec_init32(rhs, psi_out, r, xh, xl, N, nE, st))) return rc;
    if ((rc = vec_norm2(rhs, N, S->part, np_vec, st))) return rc;
    if ((rc = pcg_scalars(STAGE_FNORM, nE, S->part, np_vec, s, st))) return rc;
    if ((rc = apply_pc_mixed(Q, r, z, nullptr, S->dE, S->active, S->part, nullptr, nE, st))) return rc;
    if ((rc = pcg_scalars(STAGE_RHO, nE, S->part, np_row, s, st))) return rc;
    if ((rc = vec_p32(p, z, S->beta, S->active, N, nE, 1, st))) return rc;
    Q->launches += 5;
    const int CHECK = 4;
    for (int it = 1; it <= maxit; ++it) {
        if ((rc = apply_A_mixed(Q, p, w, S->dE, S->act32, S->act64, S->part, nE, st))) return rc;
        if ((rc = pcg_scalars(STAGE_ALPHA, nE, S->part, np_col, s, st))) return rc;
        if ((rc = vec_xr32(xh, xl, r, p, w, S->alpha, S->active, N, nE, S->part, np_vec, st))) return rc;
        if ((rc = pcg_scalars(STAGE_RNORM_RU, nE, S->part, np_vec, s, st))) return rc;
        // reliable update of the flagged energies (t is free here)
        if ((rc = vec_fold(psi_out, xh, xl, S->upd, N, nE, st))) return rc;
        if ((rc = apply_A(Q, psi_out, S->t, S->dE, S->upd, S->part2, nE, st))) return rc;
        if ((rc = vec_res32(rhs, S->t, r, S->upd, N, nE, S->part, np_vec, st))) return rc;
        if ((rc = pcg_scalars(STAGE_TRUE, nE, S->part, np_vec, s, st))) return rc;
        Q->launches += 6;
        if (it % CHECK == 0 || it == maxit) {
            int na = 0;
            if ((rc = cuda_status(cudaMemcpyAsync(&na, S->nactive, sizeof(int), cudaMemcpyDeviceToHost, st)))) return rc;
            if ((rc = cuda_status(cudaStreamSynchronize(st)))) return rc;
            if (na <= 0) break;
        }
        if (it == maxit) break;
        if ((rc = apply_pc_mixed(Q, r, z, w, S->dE, S->active, S->part, S->part2, nE, st))) return rc;
        if ((rc = pcg_scalars(STAGE_BETA_FLEX, nE, S->part, np_row, s, st, S->part2))) return rc;
        if ((rc = vec_p32(p, z, S->beta, S->active, N, nE, 0, st))) return rc;
        Q->launches += 2;
    }
    Q->launches += 1;
    return vec_fold(psi_out, xh, xl, nullptr, N, nE, st);     // energies stopped at maxit
}

static int ensure_gcr(Pcg* S, int nE) {
    if (S->gcap >= nE) return SOFT_OK;
    void* v[] = {S->gP, S->gQ, S->gbeta, S->gpart, S->gqn};
    for (void* b : v) cudaFree(b);
    S->gP = S->gQ = nullptr; S->gbeta = S->gpart = nullptr; S->gqn = nullptr;
    const size_t vb = sizeof(double2) * (size_t)S->N * nE * Pcg::GCR_M;
    int rc;
    if ((rc = cuda_status(cudaMalloc(&S->gP, vb)))) return rc;
    if ((rc = cuda_status(cudaMalloc(&S->gQ, vb)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->gbeta, sizeof(double2) * nE * Pcg::GCR_M)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->gqn, sizeof(double) * nE * Pcg::GCR_M)))) return rc;
    if ((rc = cuda_status(cudaMalloc((void**)&S->gpart, sizeof(double2) * (size_t)nE * Pcg::GCR_M * 256)))) return rc;
    S->gcap = nE;
    return SOFT_OK;
}

int pcg_refill_potential(Plan2D* Q) {
    Pcg* S = Q->pcg;
    if (!S || !S->tables) return SOFT_OK;
    int rc;
    if ((rc = refill_c(S->U, Q->U, SOFT_C128))) return rc;
    return refill_c(S->U32, Q->U, SOFT_C64);
}

void Plan2D::free_pcg() {
    delete pcg;
    pcg = nullptr;
}

}  // namespace soft

extern "C" {

static int sse_apply_A_impl(soft_plan* P, double E, const void* x, void* y, void* stream) {
    if (P && P->kind == 1 && x && y && std::isfinite(E)) return sse1d_apply(P, E, 0, 0, x, y, (cudaStream_t)stream);
    if (!P || !x || !y || P->kind != 2 || !std::isfinite(E)) return SOFT_ERR_INVALID_ARG;
    if (P->prec != SOFT_C128) return SOFT_ERR_UNSUPPORTED;
    Plan2D* Q = P->p2;
    int rc = ensure_workspace(Q, 1);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Q->launches = 0;
    if ((rc = cuda_status(cudaMemcpyAsync(Q->pcg->dE, &E, sizeof(double), cudaMemcpyHostToDevice, st))))
        return rc;
    rc = apply_A(Q, x, y, Q->pcg->dE, nullptr, Q->pcg->part, 1, st);
    P->last_launches = Q->launches;
    return rc;
}
int sse_apply_A(soft_plan* P, double E, const void* x, void* y, void* stream) {
    return abi_guard([&] { return sse_apply_A_impl(P, E, x, y, stream); });
}

static int sse_apply_A32_impl(soft_plan* P, double E, const void* x, void* y, void* stream) {
    if (P && P->kind == 1) return SOFT_ERR_UNSUPPORTED;
    if (!P || !x || !y || P->kind != 2 || !std::isfinite(E)) return SOFT_ERR_INVALID_ARG;
    if (P->prec != SOFT_C128) return SOFT_ERR_UNSUPPORTED;
    Plan2D* Q = P->p2;
    int rc = ensure_workspace(Q, 1);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Q->launches = 0;
    if ((rc = cuda_status(cudaMemcpyAsync(Q->pcg->dE, &E, sizeof(double), cudaMemcpyHostToDevice, st))))
        return rc;
    rc = apply_A_mixed(Q, x, y, Q->pcg->dE, nullptr, nullptr, Q->pcg->part, 1, st);
    P->last_launches = Q->launches;
    return rc;
}
int sse_apply_A32(soft_plan* P, double E, const void* x, void* y, void* stream) {
    return abi_guard([&] { return sse_apply_A32_impl(P, E, x, y, stream); });
}

static int sse_apply_precond_impl(soft_plan* P, double E, int precond, const void* x, void* y, void* stream) {
    if (P && P->kind == 1 && x && y && std::isfinite(E)) {
        if (precond != 0 && precond != 1 && precond != 4) return SOFT_ERR_INVALID_ARG;
        return sse1d_apply(P, E, 1, precond, x, y, (cudaStream_t)stream);
    }
    if (!P || !x || !y || P->kind != 2 || !std::isfinite(E)) return SOFT_ERR_INVALID_ARG;
    if (precond != 0 && precond != 1 && precond != 4) return SOFT_ERR_INVALID_ARG;
    if (P->prec != SOFT_C128) return SOFT_ERR_UNSUPPORTED;
    Plan2D* Q = P->p2;
    int rc = ensure_workspace(Q, 1);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Q->launches = 0;
    if ((rc = cuda_status(cudaMemcpyAsync(Q->pcg->dE, &E, sizeof(double), cudaMemcpyHostToDevice, st))))
        return rc;
    rc = apply_pc(Q, precond, x, y, Q->pcg->dE, nullptr, nullptr, 1, st);
    P->last_launches = Q->launches;
    return rc;
}
int sse_apply_precond(soft_plan* P, double E, int precond, const void* x, void* y, void* stream) {
    return abi_guard([&] { return sse_apply_precond_impl(P, E, precond, x, y, stream); });
}

static int sse_pcg_solve_impl(soft_plan* P, const double* E, int nE, const void* rhs, void* psi_out, double tol,
                              int maxit, int precond, int* iters_out, double* relres_out, void* stream) {
    if (!P || !E || nE <= 0 || !rhs || !psi_out || !(tol > 0) || maxit <= 0) return SOFT_ERR_INVALID_ARG;
    if (precond < 0 || precond > 5) return SOFT_ERR_INVALID_ARG;
    if (P->kind == 1) {                  // 1D plans: the resident solver of sse1d.cu
        for (int e = 0; e < nE; ++e)
            if (!std::isfinite(E[e])) return SOFT_ERR_INVALID_ARG;
        return sse1d_solve(P, E, nE, rhs, psi_out, tol, maxit, precond, iters_out, relres_out,
                           (cudaStream_t)stream);
    }
    const bool flexible = precond == 2 || precond == 3;
    // precond 5: the mixed iteration (solve_mixed); reliable updates after a
    // tenfold drop of the recursive residual, or after 200 iterations
    const bool mixed = precond == 5;
    const double RU_DELTA = 0.1;
    const int RU_MAXGAP = 200;
    const bool learned = precond == 2;
    if (learned) {
        if (!P->p2 || P->p2->nx % 128) return SOFT_ERR_UNSUPPORTED;
        if (nE > NN_MAX_FIELDS) return SOFT_ERR_TOO_LARGE;
        if (!P->nn) {
            P->nn = new NNState();
            int r0 = P->nn->init(1505);
            if (r0) return r0;
        }
    }
    if (flexible) precond = 1;
    if (P->kind != 2) return SOFT_ERR_INVALID_ARG;
    if (P->prec != SOFT_C128) return SOFT_ERR_UNSUPPORTED;
    for (int e = 0; e < nE; ++e)
        if (!std::isfinite(E[e])) return SOFT_ERR_INVALID_ARG;
    Plan2D* Q = P->p2;
    int rc = ensure_workspace(Q, nE);
    if (rc) return rc;
    Pcg* S = Q->pcg;
    cudaStream_t st = (cudaStream_t)stream;
    Q->launches = 0;
    const int64_t N = S->N;
    // state
    std::vector<int> ones(nE, 1), zeros(nE, 0), nconv(nE, SOFT_ERR_NOT_CONVERGED);
    std::vector<double> rel1(nE, 1.0);
    if ((rc = cuda_status(cudaMemcpy(S->dE, E, sizeof(double) * nE, cudaMemcpyHostToDevice)))) return rc;
    if ((rc = cuda_status(cudaMemcpy(S->active, ones.data(), sizeof(int) * nE, cudaMemcpyHostToDevice)))) return rc;
    if ((rc = cuda_status(cudaMemcpy(S->iters, zeros.data(), sizeof(int) * nE, cudaMemcpyHostToDevice)))) return rc;
    if ((rc = cuda_status(cudaMemcpy(S->status, nconv.data(), sizeof(int) * nE, cudaMemcpyHostToDevice)))) return rc;
    if ((rc = cuda_status(cudaMemcpy(S->nactive, &nE, sizeof(int), cudaMemcpyHostToDevice)))) return rc;
    if ((rc = cuda_status(cudaMemcpy(S->rref, rel1.data(), sizeof(double) * nE, cudaMemcpyHostToDevice)))) return rc;
    if ((rc = cuda_status(cudaMemcpy(S->upd, zeros.data(), sizeof(int) * nE, cudaMemcpyHostToDevice)))) return rc;
    if ((rc = cuda_status(cudaMemcpy(S->lastu, zeros.data(), sizeof(int) * nE, cudaMemcpyHostToDevice)))) return rc;
    if ((rc = cuda_status(cudaMemcpy(S->mode, zeros.data(), sizeof(int) * nE, cudaMemcpyHostToDevice)))) return rc;
    if ((rc = cuda_status(cudaMemcpy(S->act32, ones.data(), sizeof(int) * nE, cudaMemcpyHostToDevice)))) return rc;
    if ((rc = cuda_status(cudaMemcpy(S->act64, zeros.data(), sizeof(int) * nE, cudaMemcpyHostToDevice)))) return rc;
    PcgState s{S->rho, S->alpha, S->beta, S->relres, S->fnorm2, S->active, S->iters, S->status,
               S->nactive, tol, S->rref, S->upd, RU_DELTA, RU_MAXGAP, S->lastu,
               mixed ? S->mode : nullptr, mixed ? S->act32 : nullptr, mixed ? S->act64 : nullptr};
    const int np_vec = 256;
    if (mixed) {
        if ((rc = solve_mixed(Q, s, rhs, psi_out, maxit, nE, st))) return rc;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) return rc;
        // energies whose mixed iteration stalled even with the FP64 A (mode
        // bit 2): COCG in FP64 with the banded preconditioner, from their x
        std::vector<int> mode_h(nE), redo(nE, 0);
        if ((rc = cuda_status(cudaMemcpy(mode_h.data(), S->mode, sizeof(int) * nE, cudaMemcpyDeviceToHost)))) return rc;
        int nredo = 0;
        for (int e = 0; e < nE; ++e)
            if (mode_h[e] & 4) { redo[e] = 1; ++nredo; }
        if (nredo > 0) {
            if ((rc = cuda_status(cudaMemcpy(S->active, redo.data(), sizeof(int) * nE, cudaMemcpyHostToDevice)))) return rc;
            if ((rc = cuda_status(cudaMemcpy(S->nactive, &nredo, sizeof(int), cudaMemcpyHostToDevice)))) return rc;
            PcgState s2 = s;
            s2.mode = nullptr; s2.act32 = nullptr; s2.act64 = nullptr;
            if ((rc = solve_cocg(Q, s2, rhs, psi_out, maxit, nE, 1, true, st))) return rc;
        }
    } else if (!flexible) {
        if ((rc = solve_cocg(Q, s, rhs, psi_out, maxit, nE, precond, false, st))) return rc;
        // The recursive residual decided convergence and may have drifted
        // from f - A x.  The true residual of every converged energy is
        // evaluated in FP64 and reported; an energy whose true residual is
        // not below tol restarts from its x with r = f - A x (at most
        // VERIFY_MAXIT further iterations).
        std::vector<int> stat_h(nE), act(nE, 0), redo(nE, 0);
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) return rc;
        if ((rc = cuda_status(cudaMemcpy(stat_h.data(), S->status, sizeof(int) * nE, cudaMemcpyDeviceToHost)))) return rc;
        int nver = 0, nredo = 0;
        for (int e = 0; e < nE; ++e)
            if (stat_h[e] == SOFT_OK) { act[e] = 1; ++nver; }
        if (nver > 0) {
            if ((rc = cuda_status(cudaMemcpy(S->active, act.data(), sizeof(int) * nE, cudaMemcpyHostToDevice)))) return rc;
            std::vector<double> rel(nE, 0.0), rr(nE);
            if ((rc = true_relres(Q, rhs, psi_out, nE, act, rel, st))) return rc;
            if ((rc = cuda_status(cudaMemcpy(rr.data(), S->relres, sizeof(double) * nE, cudaMemcpyDeviceToHost)))) return rc;
            for (int e = 0; e < nE; ++e) {
                if (!act[e]) continue;
                rr[e] = rel[e];
                if (!(rel[e] < tol)) { redo[e] = 1; stat_h[e] = SOFT_ERR_NOT_CONVERGED; ++nredo; }
            }
            if ((rc = cuda_status(cudaMemcpy(S->relres, rr.data(), sizeof(double) * nE, cudaMemcpyHostToDevice)))) return rc;
        }
        if (nredo > 0) {
            constexpr int VERIFY_MAXIT = 50;
            if ((rc = cuda_status(cudaMemcpy(S->active, redo.data(), sizeof(int) * nE, cudaMemcpyHostToDevice)))) return rc;
            if ((rc = cuda_status(cudaMemcpy(S->status, stat_h.data(), sizeof(int) * nE, cudaMemcpyHostToDevice)))) return rc;
            if ((rc = cuda_status(cudaMemcpy(S->nactive, &nredo, sizeof(int), cudaMemcpyHostToDevice)))) return rc;
            if ((rc = solve_cocg(Q, s, rhs, psi_out, VERIFY_MAXIT, nE, precond, true, st))) return rc;
        }
    } else {
        // x = 0, r = f, ||f||^2
        if ((rc = vec_init(rhs, psi_out, S->r, N, nE, st))) return rc;
        if ((rc = vec_norm2(rhs, N, S->part, np_vec, st))) return rc;
        if ((rc = pcg_scalars(STAGE_FNORM, nE, S->part, np_vec, s, st))) return rc;
        // flexible GCR with the last GCR_M direction pairs (minimal residual,
        // valid for a preconditioner that changes from one iteration to the
        // next, e.g. the learned correction)
        if ((rc = ensure_gcr(S, nE))) return rc;
        const int M = Pcg::GCR_M;
        const int64_t ss = N * nE;
        double2* gPb = (double2*)S->gP;
        double2* gQb = (double2*)S->gQ;
        const int CHECK = 4;
        for (int it = 1; it <= maxit; ++it) {
            const int slot = (it - 1) % M, mu = std::min(it, M);
            double2* Ps = gPb + slot * ss;
            double2* Qs = gQb + slot * ss;
            if ((rc = apply_pc(Q, precond, S->r, Ps, S->dE, S->active, nullptr, nE, st))) return rc;
            if (learned && (rc = P->nn->correct_c128(Ps, nE, Q->ny, Q->nx, S->active, st))) return rc;
            if ((rc = apply_A(Q, Ps, Qs, S->dE, S->active, S->part, nE, st))) return rc;
            if ((rc = gcr_step(0, gPb, gQb, ss, mu, M, slot, S->gbeta, S->gqn, S->r, S->active, N, nE,
                               S->gpart, S->part, S->part2, np_vec, s, st))) return rc;
            if ((rc = vec_xr(psi_out, S->r, Ps, Qs, S->alpha, S->active, N, nE, S->part, np_vec, st))) return rc;
            if ((rc = pcg_scalars(STAGE_RNORM, nE, S->part, np_vec, s, st))) return rc;
            Q->launches += (learned ? 4 : 0) + 3 + 2 + 4 + 2;
            if (it % CHECK == 0 || it == maxit) {
                int na = 0;
                if ((rc = cuda_status(cudaMemcpyAsync(&na, S->nactive, sizeof(int), cudaMemcpyDeviceToHost, st)))) return rc;
                if ((rc = cuda_status(cudaStreamSynchronize(st)))) return rc;
                if (na <= 0) break;
            }
        }
    }
    std::vector<int> it_h(nE), stat_h(nE);
    std::vector<double> rr_h(nE);
    if ((rc = cuda_status(cudaMemcpyAsync(it_h.data(), S->iters, sizeof(int) * nE, cudaMemcpyDeviceToHost, st)))) return rc;
    if ((rc = cuda_status(cudaMemcpyAsync(stat_h.data(), S->status, sizeof(int) * nE, cudaMemcpyDeviceToHost, st)))) return rc;
    if ((rc = cuda_status(cudaMemcpyAsync(rr_h.data(), S->relres, sizeof(double) * nE, cudaMemcpyDeviceToHost, st)))) return rc;
    if ((rc = cuda_status(cudaStreamSynchronize(st)))) return rc;
    P->last_launches = Q->launches;
    if (iters_out) std::memcpy(iters_out, it_h.data(), sizeof(int) * nE);
    if (relres_out) std::memcpy(relres_out, rr_h.data(), sizeof(double) * nE);
    int out = SOFT_OK;
    for (int e = 0; e < nE; ++e) {
        if (stat_h[e] == SOFT_ERR_BREAKDOWN || stat_h[e] == SOFT_ERR_NONFINITE) return stat_h[e];
        if (stat_h[e] != SOFT_OK) out = SOFT_ERR_NOT_CONVERGED;
    }
    return out;
}
int sse_pcg_solve(soft_plan* P, const double* E, int nE, const void* rhs, void* psi_out, double tol,
                  int maxit, int precond, int* iters_out, double* relres_out, void* stream) {
    return abi_guard([&] { return sse_pcg_solve_impl(P, E, nE, rhs, psi_out, tol, maxit, precond, iters_out, relres_out, stream); });
}

}  // extern "C"
