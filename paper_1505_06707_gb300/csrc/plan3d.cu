// 3D plans: host FP64 tables for a [nz][ny][nx] grid and the step driver.
//
// The scheme is the one printed after Eq. C_FD (Sec. II) with
// K = (kx^2 + ky^2 + kz^2)/2 and C = C_x + C_y + C_z as Kronecker sums (the
// multidimensional case named at the end of Sec. V).  In time order the
// merged scheme is ... V/2, CN, V/2, K ... with V/2 = e^{-iU tau/2}; factors
// on different axes commute, so one step is four passes over the grid, the
// state kept in x space between them:
//   X  rows (x lines):     K_x, V/2, CN_x (and the second V/2 on the rows
//                          outside the y- and z-strip blocks)
//   Y1 y-strip block:      CN_y
//   Z  z lines:            CN_z, V/2 (on the points not done by X), K_z
//   Y2 y lines:            K_y
// which is K_x | V/2 CN_x CN_y CN_z V/2 | K_z K_y per step; a call starts
// with K_y/2, K_z/2 and ends with K_x/2, and the first and last steps use
// the half factors K_x/2 and K_z/2, K_y/2.  The middle steps are replayed
// from a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>

#include "plan_internal.h"
#include "soft2d.cuh"

using namespace soft;

namespace soft {

static int ilog2_3d(int64_t n) {
    int l = 0;
    while ((int64_t(1) << l) < n) ++l;
    return (int64_t(1) << l) == n ? l : -1;
}

Plan3D::~Plan3D() {
    void* bufs[] = {W[0], W[1], W[2], TK[0], TK[1], TK[2], TKh[0], TKh[1], TKh[2],
                    TVh, cn[0], cn[1], cn[2]};
    for (void* b : bufs) cudaFree(b);
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
}

// e^{-iU tau/2} from U (host [nz][ny][nx]) plus the axes' absorber terms;
// z planes are split over host threads (512^3 points take seconds alone)
static std::vector<cd> half_factors(const Plan3D& Q, const double* Uin) {
    const int nx = Q.n[0], ny = Q.n[1], nz = Q.n[2];
    std::vector<cd> tvh((size_t)nx * ny * nz);
    auto planes = [&](int z0, int z1) {
        for (int z = z0; z < z1; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const size_t i = ((size_t)z * ny + y) * nx + x;
                    cd u;
                    if (Uin) {
                        u = cd(Uin[2 * i], Uin[2 * i + 1]);
                    } else {
                        const cd zz[3] = {Q.ax[0].z[x], Q.ax[1].z[y], Q.ax[2].z[z]};
                        u = soft_coulomb(zz, 3, Q.a2, Q.charge);
                    }
                    u += Q.ua[0][x] + Q.ua[1][y] + Q.ua[2][z];
                    tvh[i] = std::exp(cd(0.0, -0.5 * Q.tau) * u);
                }
    };
    const int nt = std::max(1, std::min({(int)std::thread::hardware_concurrency(), 32, nz}));
    std::vector<std::thread> pool;
    int done = 0;                  // planes handed to threads; the rest run here
    try {
        for (int t = 0; t < nt; ++t) {
            const int z0 = (int)((int64_t)nz * t / nt), z1 = (int)((int64_t)nz * (t + 1) / nt);
            pool.emplace_back(planes, z0, z1);
            done = z1;
        }
    } catch (...) {                // no thread could be started: no exception crosses the C ABI
    }
    for (auto& th : pool) th.join();
    if (done < nz) planes(done, nz);
    return tvh;
}

int Plan3D::set_potential(const double* Uin) {
    int rc = cuda_status(cudaDeviceSynchronize());      // no step may still read the table
    if (rc) return rc;
    return refill_vtab(TVh, half_factors(*this, Uin), prec);
}

int Plan3D::row(int mode, void* psi, const void* tkx, cudaStream_t st) {
    ++launches;
    const int nrows = n[1] * n[2];
    if (prec == SOFT_C64) return soft2d_row_c64(l[0], le[0], lr[0], mode, geo, psi, nrows, tkx, st);
    return soft2d_row_c128(l[0], le[0], lr[0], mode, geo, psi, nrows, tkx, st);
}

// a line pass along axis d = 1, 2 (COL_K, or COL_CVK with the axis' strip CN
// and V/2)
int Plan3D::line(int d, int mode, void* psi, const void* tk, cudaStream_t st) {
    ++launches;
    const int64_t nx = n[0], ny = n[1];
    // z lines (c = y nx + x): V/2 off the z-strip block only on lines with y
    // in the y-strip block (the row pass applied it on the others)
    const LineGeo lg{W[d], d == 1 ? nx : nx * ny, d == 1 ? nx * ny : 0, cn[d], TVh, nb[d], blk0[d],
                     d == 2 ? nx : 0, n[1], nb[1], blk0[1]};
    const int planes = d == 1 ? n[2] : 1;
    if (prec == SOFT_C64) return soft2d_col_c64(l[d], le[d], lr[d], mode, lg, planes, psi, tk, st);
    return soft2d_col_c128(l[d], le[d], lr[d], mode, lg, planes, psi, tk, st);
}

// CN on the strip block of every line along axis d = 1, 2
int Plan3D::cnpass(int d, void* psi, cudaStream_t st) {
    if (nb[d] == 0) return SOFT_OK;
    ++launches;
    const int64_t nx = n[0], ny = n[1];
    const CnGeo cg{cn[d], nb[d], blk0[d], n[d], d == 1 ? nx : nx * ny, d == 1 ? nx * ny : 0};
    const int planes = d == 1 ? n[2] : 1;
    if (prec == SOFT_C64) return soft2d_cny_c64(cg, planes, psi, st);
    return soft2d_cny_c128(cg, planes, psi, st);
}

int Plan3D::col_capacity(int d) const {
    return prec == SOFT_C64 ? soft2d_col_strip_capacity_c64(l[d], le[d], lr[d])
                            : soft2d_col_strip_capacity_c128(l[d], le[d], lr[d]);
}

// one step: X (K_x, V/2, CN_x), Y1 (CN_y), Z (CN_z, V/2, K_z), Y2 (K_y); the
// first step of a call takes K_x/2, the last K_z/2 and K_y/2
int Plan3D::enqueue_step(void* psi, bool first, bool last, cudaStream_t st) {
    int rc;
    if ((rc = row(ROW_KVC, psi, first ? TKh[0] : TK[0], st))) return rc;
    if ((rc = cnpass(1, psi, st))) return rc;
    if ((rc = line(2, COL_CVK, psi, last ? TKh[2] : TK[2], st))) return rc;
    return line(1, COL_K, psi, last ? TKh[1] : TK[1], st);
}

}  // namespace soft

int create_3d(const soft_grid* grid, const double* box, double R0, double theta, double dt,
              const soft_options& o, soft_plan** out) {
    int ln[3];
    for (int d = 0; d < 3; ++d) {
        ln[d] = ilog2_3d(grid->n[d]);
        if (ln[d] < 6 || ln[d] > 11) return SOFT_ERR_NOT_POW2;
        const double a = box[2 * d], b = box[2 * d + 1];
        if (!(b > 0) || std::fabs(a + b) > 1e-12 * b || !(R0 > 0 && R0 < b)) return SOFT_ERR_INVALID_ARG;
    }
    if (grid->n[1] * grid->n[2] > 0x7fffffff / 2) return SOFT_ERR_TOO_LARGE;
    std::unique_ptr<soft_plan> P(new soft_plan());
    P->kind = 3;
    P->prec = o.prec;
    P->opt = o;
    P->dt = dt;
    Plan3D* Q = new Plan3D();
    P->p3 = Q;
    Q->prec = o.prec;
    Q->tau = dt;
    Q->a2 = o.soft_a2;
    Q->charge = o.charge;
    for (int d = 0; d < 3; ++d) {
        Q->n[d] = (int)grid->n[d];
        Q->l[d] = ln[d];
        soft1d_default_cfg(o.prec, ln[d], &Q->le[d], &Q->lr[d]);
    }
    // line passes: 32 elements per thread in complex64 (as the 2D column pass)
    for (int d = 1; d < 3; ++d)
        if (o.prec == SOFT_C64 && ln[d] >= 10) Q->le[d] = 5;
    int rc;
    for (int d = 0; d < 3; ++d) {
        ContourFn cf(o.contour, R0, box[2 * d + 1], theta, o.tfecs_alpha, o.cap_energy, o.tfap_kmin);
        build_axis(Q->ax[d], Q->n[d], box[2 * d], box[2 * d + 1], cf, dt);
        Q->ua[d].resize(Q->n[d]);
        for (int i = 0; i < Q->n[d]; ++i) Q->ua[d][i] = cf.absorber(Q->ax[d].x[i]);
        if ((rc = find_block(Q->ax[d], &Q->blk0[d], &Q->nb[d]))) return rc;
    }
    // strip rows per thread of the row pass, of the y-strip CN pass (a tile
    // of at least 32 lines and the LU coefficients in shared memory) and of
    // the z line pass
    const int thr = Q->n[0] >> Q->le[0];
    if ((Q->nb[0] + thr - 1) / thr > (1 << Q->le[0]) / 4 + 2) return SOFT_ERR_UNSUPPORTED;
    if ((o.prec == SOFT_C64 ? 8 : 16) * (size_t)Q->nb[1] * 35 > 227 * 1024) return SOFT_ERR_UNSUPPORTED;
    if (Q->nb[2] > Q->col_capacity(2)) return SOFT_ERR_UNSUPPORTED;
    // kinetic factors per axis, 1/n folded in, in the transposed order of
    // the fused center of each line FFT
    auto ktab = [&](int d, double frac) {
        const Axis1D& A = Q->ax[d];
        const int logn = Q->l[d], logrm = Q->lr[d];
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
    const int pr = o.prec;
    for (int d = 0; d < 3; ++d) {
        if ((rc = upload_tw(&Q->W[d], pr == SOFT_C128 ? pass_twiddles_full(Q->l[d], Q->lr[d], TWFULL_MAXS)
                                                     : pass_twiddles(Q->l[d], Q->lr[d]), pr)))
            return rc;
        if ((rc = upload_tab(&Q->TK[d], ktab(d, 1.0), pr))) return rc;
        if ((rc = upload_tab(&Q->TKh[d], ktab(d, 0.5), pr))) return rc;
        if (Q->nb[d] > 0) {
            std::vector<cd> mf, mb, g;
            double err;
            if ((rc = strip_factor(Q->ax[d], Q->blk0[d], Q->nb[d], mf, mb, g, &err))) return rc;
            mf.insert(mf.end(), mb.begin(), mb.end());
            mf.insert(mf.end(), g.begin(), g.end());
            if ((rc = upload_c(&Q->cn[d], mf, pr))) return rc;
        }
    }
    if ((rc = upload_vtab(&Q->TVh, half_factors(*Q, nullptr), pr))) return rc;
    Geo2D& g = Q->geo;
    std::memset(&g, 0, sizeof(g));
    g.Wx = Q->W[0]; g.TVh = Q->TVh; g.cnx = Q->cn[0];
    g.nx = Q->n[0]; g.ny = Q->n[1] * Q->n[2];
    g.nbx = Q->nb[0]; g.blk0x = Q->blk0[0];
    g.nby = Q->nb[1]; g.blk0y = Q->blk0[1];
    g.v2 = 1; g.ny1 = Q->n[1]; g.nz1 = Q->n[2]; g.nbz1 = Q->nb[2]; g.blk0z1 = Q->blk0[2];
    // set every kernel's shared-memory attribute now, outside any stream capture
    for (int m = ROW_K; m <= ROW_KVC; ++m)
        if ((rc = Q->row(m, nullptr, nullptr, 0))) return rc;
    for (int d = 1; d < 3; ++d)
        for (int m = COL_K; m <= COL_CVK; ++m)
            if ((rc = Q->line(d, m, nullptr, nullptr, 0))) return rc;
    if ((rc = Q->cnpass(1, nullptr, 0))) return rc;
    Q->launches = 0;
    *out = P.release();
    return SOFT_OK;
}

// The call: K_y/2 and K_z/2 (line passes), n steps (the first with K_x/2,
// the last with K_z/2 and K_y/2), then K_x/2 (row pass).
int soft_plan::step_3d(void* psi, int64_t nsteps, double* t_inout, cudaStream_t st) {
    Plan3D* Q = p3;
    Q->launches = 0;
    last_launches = 0;
    if (nsteps == 0) return SOFT_OK;
    int rc;
    if ((rc = Q->line(1, COL_K, psi, Q->TKh[1], st))) return rc;
    if ((rc = Q->line(2, COL_K, psi, Q->TKh[2], st))) return rc;
    if ((rc = Q->enqueue_step(psi, true, nsteps == 1, st))) return rc;
    int64_t mid = nsteps >= 2 ? nsteps - 2 : 0;
    const int64_t G = Plan3D::GRAPH_STEPS;
    if (mid >= G) {
        if (!Q->graph_exec || Q->graph_psi != psi || Q->graph_stream != st) {
            if (Q->graph_exec) { cudaGraphExecDestroy(Q->graph_exec); Q->graph_exec = nullptr; }
            cudaStream_t cap;
            if ((rc = cuda_status(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)))) return rc;
            cudaGraph_t graph;
            const int64_t before = Q->launches;
            rc = cuda_status(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
            for (int64_t s = 0; s < G && rc == SOFT_OK; ++s) rc = Q->enqueue_step(psi, false, false, cap);
            cudaError_t e = cudaStreamEndCapture(cap, &graph);
            if (rc == SOFT_OK) rc = cuda_status(e);
            if (rc == SOFT_OK) rc = cuda_status(cudaGraphInstantiate(&Q->graph_exec, graph, 0));
            if (e == cudaSuccess) cudaGraphDestroy(graph);
            cudaStreamDestroy(cap);
            if (rc) { Q->graph_exec = nullptr; return rc; }
            Q->graph_psi = psi;
            Q->graph_stream = st;
            Q->graph_launches = Q->launches - before;
            Q->launches = before;
        }
        while (mid >= G) {
            if ((rc = cuda_status(cudaGraphLaunch(Q->graph_exec, st)))) return rc;
            Q->launches += Q->graph_launches;
            mid -= G;
        }
    }
    for (int64_t s = 0; s < mid; ++s)
        if ((rc = Q->enqueue_step(psi, false, false, st))) return rc;
    if (nsteps >= 2 && (rc = Q->enqueue_step(psi, false, true, st))) return rc;
    if ((rc = Q->row(ROW_K, psi, Q->TKh[0], st))) return rc;
    last_launches = Q->launches;
    *t_inout += (double)nsteps * dt;
    return SOFT_OK;
}

int64_t soft_plan::points_3d() const { return p3 ? (int64_t)p3->n[0] * p3->n[1] * p3->n[2] : 0; }
void soft_plan::free_3d() { delete p3; p3 = nullptr; }
