// 2D plans: host FP64 tables for a [ny][nx] grid and the step driver (a row
// pass and a column pass per step, replayed from a CUDA graph).  The
// stationary PCG entry points live in pcg.cu.
#include <cmath>
#include <cstring>

#include "plan_internal.h"
#include "soft2d.cuh"

using namespace soft;

namespace soft {

static int ilog2_2d(int64_t n) {
    int l = 0;
    while ((int64_t(1) << l) < n) ++l;
    return (int64_t(1) << l) == n ? l : -1;
}

// replace the potential (host complex [ny][nx], plus the plan's absorber
// part) and rewrite e^{-iU tau/2} and the solver's U tables in place
int Plan2D::set_potential(const double* Uin) {
    int rc = cuda_status(cudaDeviceSynchronize());      // no step may still read the tables
    if (rc) return rc;
    const size_t n = (size_t)nx * ny;
    std::vector<cd> tvh(n);
    for (size_t i = 0; i < n; ++i) {
        U[i] = cd(Uin[2 * i], Uin[2 * i + 1]) + Uabs[i];
        tvh[i] = std::exp(cd(0.0, -0.5 * tau) * U[i]);
    }
    if ((rc = refill_vtab(TVh, tvh, prec))) return rc;
    return pcg_refill_potential(this);
}

Plan2D::~Plan2D() {
    void* bufs[] = {Wx, Wy, TKx, TKhx, TKy, TKhy, TVh, cnx, cny};
    for (void* b : bufs) cudaFree(b);
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    free_pcg();
}

int Plan2D::row(int mode, void* psi, const void* tkx, cudaStream_t st) {
    ++launches;
    if (prec == SOFT_C64) return soft2d_row_c64(lx, lex, lrx, mode, geo, psi, ny, tkx, st);
    return soft2d_row_c128(lx, lex, lrx, mode, geo, psi, ny, tkx, st);
}
int Plan2D::col(int mode, void* psi, const void* tky, cudaStream_t st) {
    ++launches;
    const LineGeo lg{geo.Wy, geo.nx, 0, geo.cny, geo.TVh, geo.nby, geo.blk0y, 0, 1, 0, 0};
    if (prec == SOFT_C64) return soft2d_col_c64(ly, ley, lry, mode, lg, 1, psi, tky, st);
    return soft2d_col_c128(ly, ley, lry, mode, lg, 1, psi, tky, st);
}

// one step in x space: row pass K_x, V/2, CN_x (and the second V/2 off the
// y-strip block); column pass CN_y, V/2 on the block rows, K_y
int Plan2D::enqueue_step(void* psi, const void* tkx, const void* tky, cudaStream_t st) {
    int rc;
    if ((rc = row(ROW_KVC, psi, tkx, st))) return rc;
    return col(COL_CBK, psi, tky, st);
}

}  // namespace soft

int create_2d(const soft_grid* grid, const double* box, double R0, double theta, double dt,
              const soft_options& o, soft_plan** out) {
    const int64_t nx = grid->n[0], ny = grid->n[1];
    const int lx = ilog2_2d(nx), ly = ilog2_2d(ny);
    if (lx < 8 || lx > 11 || ly < 8 || ly > 11) return SOFT_ERR_NOT_POW2;
    for (int d = 0; d < 2; ++d) {
        const double a = box[2 * d], b = box[2 * d + 1];
        if (!(b > 0) || std::fabs(a + b) > 1e-12 * b || !(R0 > 0 && R0 < b)) return SOFT_ERR_INVALID_ARG;
    }
    std::unique_ptr<soft_plan> P(new soft_plan());
    P->kind = 2;
    P->prec = o.prec;
    P->opt = o;
    P->dt = dt;
    Plan2D* Q = new Plan2D();
    P->p2 = Q;
    Q->prec = o.prec;
    Q->nx = (int)nx; Q->ny = (int)ny;
    Q->lx = lx; Q->ly = ly;
    soft1d_default_cfg(o.prec, lx, &Q->lex, &Q->lrx);
    soft1d_default_cfg(o.prec, ly, &Q->ley, &Q->lry);
    // column pass: 32 elements per thread in complex64 (two CTAs of 4 columns per SM)
    if (o.prec == SOFT_C64 && ly >= 10) Q->ley = 5;
    Q->R0 = R0; Q->theta = theta; Q->tau = dt;
    Q->band_width = o.band_width;
    ContourFn cx(o.contour, R0, box[1], theta, o.tfecs_alpha, o.cap_energy, o.tfap_kmin);
    ContourFn cy(o.contour, R0, box[3], theta, o.tfecs_alpha, o.cap_energy, o.tfap_kmin);
    build_axis(Q->ax, (int)nx, box[0], box[1], cx, dt);
    build_axis(Q->ay, (int)ny, box[2], box[3], cy, dt);
    int rc;
    int bx0, nbx, by0, nby;
    if ((rc = find_block(Q->ax, &bx0, &nbx))) return rc;
    if ((rc = find_block(Q->ay, &by0, &nby))) return rc;
    // strip rows per thread of the row pass and of the column pass
    const int thr = (int)(nx >> Q->lex);
    if ((nbx + thr - 1) / thr > (1 << Q->lex) / 4 + 2) return SOFT_ERR_UNSUPPORTED;
    const int capy = o.prec == SOFT_C64 ? soft2d_col_strip_capacity_c64(ly, Q->ley, Q->lry)
                                        : soft2d_col_strip_capacity_c128(ly, Q->ley, Q->lry);
    if (nby > capy) return SOFT_ERR_UNSUPPORTED;
    // potential at (z(x), z(y)) and e^{-iU tau/2}
    Q->U.resize((size_t)nx * ny);
    Q->Uabs.resize((size_t)nx * ny);
    std::vector<cd> tvh((size_t)nx * ny);
    for (int64_t yy = 0; yy < ny; ++yy)
        for (int64_t xx = 0; xx < nx; ++xx) {
            const cd z[2] = {Q->ax.z[xx], Q->ay.z[yy]};
            const cd ua = cx.absorber(Q->ax.x[xx]) + cy.absorber(Q->ay.x[yy]);
            const cd u = soft_coulomb(z, 2, o.soft_a2, o.charge) + ua;
            Q->Uabs[yy * nx + xx] = ua;
            Q->U[yy * nx + xx] = u;
            tvh[yy * nx + xx] = std::exp(cd(0.0, -0.5 * dt) * u);
        }
    // kinetic factors per axis, 1/n folded in, read by the fused center of
    // each line FFT (butterflies of R consecutive positions b*R + m of the
    // digit-reversed spectrum, stored at m*(n/R) + b)
    auto ktab = [&](const Axis1D& A, int logn, int logrm, double frac) {
        const std::vector<int> perm = dif_output_order(logn, logrm);
        const int lrl = (logn % logrm) ? logn % logrm : logrm;
        const int Rl = 1 << lrl, nbf = A.n >> lrl;
        std::vector<cd> t(A.n);
        for (int p = 0; p < A.n; ++p) {
            const double k = A.k[perm[p]];
            const int q = (p % Rl) * nbf + p / Rl;
            t[q] = std::polar(1.0 / A.n, -0.5 * k * k * dt * frac);
        }
        return t;
    };
    std::vector<cd> mfx, mbx, gx, mfy, mby, gy, cnx, cny;
    double err;
    if (nbx > 0) {
        if ((rc = strip_factor(Q->ax, bx0, nbx, mfx, mbx, gx, &err))) return rc;
        cnx = mfx; cnx.insert(cnx.end(), mbx.begin(), mbx.end()); cnx.insert(cnx.end(), gx.begin(), gx.end());
    }
    if (nby > 0) {
        if ((rc = strip_factor(Q->ay, by0, nby, mfy, mby, gy, &err))) return rc;
        cny = mfy; cny.insert(cny.end(), mby.begin(), mby.end()); cny.insert(cny.end(), gy.begin(), gy.end());
    }
    const int pr = o.prec;
    // pass twiddles: the four bases per pass (complex64); every W^{M off} of
    // the small-stride passes (complex128)
    auto twid = [&](void** d, int logn, int logrm) {
        return upload_tw(d, pr == SOFT_C128 ? pass_twiddles_full(logn, logrm, TWFULL_MAXS)
                                            : pass_twiddles(logn, logrm), pr);
    };
    if ((rc = twid(&Q->Wx, lx, Q->lrx))) return rc;
    if ((rc = twid(&Q->Wy, ly, Q->lry))) return rc;
    if ((rc = upload_tab(&Q->TKx, ktab(Q->ax, lx, Q->lrx, 1.0), pr))) return rc;
    if ((rc = upload_tab(&Q->TKhx, ktab(Q->ax, lx, Q->lrx, 0.5), pr))) return rc;
    if ((rc = upload_tab(&Q->TKy, ktab(Q->ay, ly, Q->lry, 1.0), pr))) return rc;
    if ((rc = upload_tab(&Q->TKhy, ktab(Q->ay, ly, Q->lry, 0.5), pr))) return rc;
    if ((rc = upload_vtab(&Q->TVh, tvh, pr))) return rc;
    if ((rc = upload_c(&Q->cnx, cnx, pr))) return rc;
    if ((rc = upload_c(&Q->cny, cny, pr))) return rc;
    Geo2D& g = Q->geo;
    g.Wx = Q->Wx; g.Wy = Q->Wy; g.TVh = Q->TVh; g.cnx = Q->cnx; g.cny = Q->cny;
    g.nx = (int)nx; g.ny = (int)ny;
    g.nbx = nbx; g.blk0x = bx0; g.nby = nby; g.blk0y = by0;
    g.v2 = 1; g.ny1 = (int)ny; g.nz1 = 1; g.nbz1 = 0; g.blk0z1 = 0;
    // set every kernel's shared-memory attribute now, outside any stream capture
    for (int m = ROW_K; m <= ROW_KVC; ++m)
        if ((rc = Q->row(m, nullptr, nullptr, 0))) return rc;
    for (int m = COL_K; m <= COL_CBK; ++m)
        if ((rc = Q->col(m, nullptr, nullptr, 0))) return rc;
    Q->launches = 0;
    *out = P.release();
    return SOFT_OK;
}

// The call in time order: K_y/2 (column pass), then n steps of [row pass
// K_x, V/2, CN_x; column pass CN_y, V/2, K_y] with K_x/2 in the first row
// pass and K_y/2 in the last column pass, then K_x/2 (row pass): the
// printed K/2 V/2 CN V/2 K/2 per step with the inner half-kinetic factors
// merged.  The middle steps are replayed from a CUDA graph captured once per
// state pointer and stream (chunks of GRAPH_STEPS steps).
int soft_plan::step_2d(void* psi, int64_t nsteps, double* t_inout, cudaStream_t st) {
    Plan2D* Q = p2;
    Q->launches = 0;
    last_launches = 0;
    if (nsteps == 0) return SOFT_OK;
    int rc;
    if ((rc = Q->col(COL_K, psi, Q->TKhy, st))) return rc;
    if ((rc = Q->enqueue_step(psi, Q->TKhx, nsteps == 1 ? Q->TKhy : Q->TKy, st))) return rc;
    int64_t mid = nsteps >= 2 ? nsteps - 2 : 0;
    const int64_t G = Plan2D::GRAPH_STEPS;
    if (mid >= G) {
        if (!Q->graph_exec || Q->graph_psi != psi || Q->graph_stream != st) {
            if (Q->graph_exec) { cudaGraphExecDestroy(Q->graph_exec); Q->graph_exec = nullptr; }
            cudaStream_t cap;
            if ((rc = cuda_status(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)))) return rc;
            cudaGraph_t graph;
            const int64_t before = Q->launches;
            rc = cuda_status(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
            for (int64_t s = 0; s < G && rc == SOFT_OK; ++s) rc = Q->enqueue_step(psi, Q->TKx, Q->TKy, cap);
            cudaError_t e = cudaStreamEndCapture(cap, &graph);
            if (rc == SOFT_OK) rc = cuda_status(e);
            if (rc == SOFT_OK) rc = cuda_status(cudaGraphInstantiate(&Q->graph_exec, graph, 0));
            if (e == cudaSuccess) cudaGraphDestroy(graph);
            cudaStreamDestroy(cap);
            if (rc) { Q->graph_exec = nullptr; return rc; }
            Q->graph_psi = psi;
            Q->graph_stream = st;
            Q->graph_launches = Q->launches - before;   // kernels in one replay
            Q->launches = before;
        }
        while (mid >= G) {
            if ((rc = cuda_status(cudaGraphLaunch(Q->graph_exec, st)))) return rc;
            Q->launches += Q->graph_launches;
            mid -= G;
        }
    }
    for (int64_t s = 0; s < mid; ++s)
        if ((rc = Q->enqueue_step(psi, Q->TKx, Q->TKy, st))) return rc;
    if (nsteps >= 2 && (rc = Q->enqueue_step(psi, Q->TKx, Q->TKhy, st))) return rc;
    if ((rc = Q->row(ROW_K, psi, Q->TKhx, st))) return rc;
    last_launches = Q->launches;
    *t_inout += (double)nsteps * dt;
    return SOFT_OK;
}

int64_t soft_plan::points_2d() const { return p2 ? (int64_t)p2->nx * p2->ny : 0; }
void soft_plan::free_2d() { delete p2; p2 = nullptr; }
