// The opaque plan object behind the C ABI.
#pragma once
#include <memory>
#include <vector>

#include "internal.h"

#include <new>

namespace soft {
int cuda_status(cudaError_t e);
// Runs an entry point's body so that no C++ exception crosses the C ABI: a
// failed host allocation returns SOFT_ERR_OOM, any other exception
// SOFT_ERR_SETUP.
template <class F>
int abi_guard(F&& f) noexcept {
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return SOFT_ERR_OOM;
    } catch (...) {
        return SOFT_ERR_SETUP;
    }
}
int upload(void** dst, const void* src, size_t bytes);
int upload_c(void** dst, const std::vector<cd>& v, int prec);
int upload_tab(void** dst, const std::vector<cd>& v, int prec);
int upload_vtab(void** dst, const std::vector<cd>& v, int prec);
int upload_tw(void** dst, const std::vector<cd>& v, int prec);
int upload_tw_comp(void** dst, const std::vector<cd>& v, int prec);
// rewrite an existing device buffer in place (same size and format as the
// matching upload_*), so that pointers held by kernels and graphs stay valid
int refill_c(void* dst, const std::vector<cd>& v, int prec);
int refill_vtab(void* dst, const std::vector<cd>& v, int prec);
struct Plan2D;
int pcg_refill_potential(Plan2D* Q);     // the stationary solver's U tables, if built
int make_tables_1d(Tables1D* T, int n, double a, double b, double R0, double theta, double tau,
                   const soft_options& o, int loge, int logrm);

struct Geo2D;
struct NNState;
struct Sse1D;
void sse1d_free(Sse1D* s);
struct Surf1D;
void surf1d_free(Surf1D* s);
int sse1d_refill_potential(soft_plan* P);
int sse1d_solve(soft_plan* P, const double* E, int nE, const void* rhs, void* psi_out, double tol, int maxit,
                int precond, int* iters_out, double* relres_out, cudaStream_t st);
int sse1d_apply(soft_plan* P, double E, int what, int precond, const void* x, void* y, cudaStream_t st);
}  // namespace soft

#include "soft2d_geo.h"

namespace soft {
// pass kernels of the 2D and 3D steps (soft2d_c64.cu, soft2d_c128.cu)
int soft2d_row_c64(int, int, int, int, const Geo2D&, void*, int, const void*, cudaStream_t);
int soft2d_row_c128(int, int, int, int, const Geo2D&, void*, int, const void*, cudaStream_t);
int soft2d_col_c64(int, int, int, int, const LineGeo&, int, void*, const void*, cudaStream_t);
int soft2d_col_c128(int, int, int, int, const LineGeo&, int, void*, const void*, cudaStream_t);
int soft2d_col_strip_capacity_c64(int, int, int);
int soft2d_col_strip_capacity_c128(int, int, int);
int soft2d_cny_c64(const CnGeo&, int, void*, cudaStream_t);
int soft2d_cny_c128(const CnGeo&, int, void*, cudaStream_t);

// 2D plan state (plan2d.cu) and the stationary solver workspace (pcg.cu)
struct Plan2D {
    static constexpr int64_t GRAPH_STEPS = 16;
    int prec = SOFT_C128;
    int nx = 0, ny = 0, lx = 0, ly = 0, lex = 0, lrx = 0, ley = 0, lry = 0;
    int band_width = 10;
    double R0 = 0, theta = 0, tau = 0;
    Axis1D ax, ay;                 // host FP64 axes (grid, k, q, z, C)
    std::vector<cd> U;             // U(z(x), z(y)), [ny][nx]
    std::vector<cd> Uabs;          // its comparison-absorber part, [ny][nx]
    void *Wx = nullptr, *Wy = nullptr, *TKx = nullptr, *TKhx = nullptr, *TKy = nullptr,
         *TKhy = nullptr, *TVh = nullptr, *cnx = nullptr, *cny = nullptr;
    Geo2D geo{};
    int64_t launches = 0, graph_launches = 0;
    cudaGraphExec_t graph_exec = nullptr;
    void* graph_psi = nullptr;
    cudaStream_t graph_stream = nullptr;
    struct Pcg* pcg = nullptr;

    int row(int mode, void* psi, const void* tkx, cudaStream_t st);
    int col(int mode, void* psi, const void* tky, cudaStream_t st);
    int enqueue_step(void* psi, const void* tkx, const void* tky, cudaStream_t st);
    void free_pcg();
    int set_potential(const double* U_re_im);   // host complex [ny][nx]
    ~Plan2D();
};

// 3D plan state (plan3d.cu): a [nz][ny][nx] grid stepped by the line pass
// kernels (rows; lines along y and z; strip CN along y)
struct Plan3D {
    static constexpr int64_t GRAPH_STEPS = 8;
    int prec = SOFT_C128;
    int n[3] = {}, l[3] = {}, le[3] = {}, lr[3] = {};
    int nb[3] = {}, blk0[3] = {};  // strip block of each axis
    double tau = 0, a2 = 2.0, charge = 1.0;
    Axis1D ax[3];
    std::vector<cd> ua[3];         // comparison-absorber potential of each axis
    void *W[3] = {}, *TK[3] = {}, *TKh[3] = {}, *TVh = nullptr, *cn[3] = {};
    Geo2D geo{};
    int64_t launches = 0, graph_launches = 0;
    cudaGraphExec_t graph_exec = nullptr;
    void* graph_psi = nullptr;
    cudaStream_t graph_stream = nullptr;

    int row(int mode, void* psi, const void* tkx, cudaStream_t st);
    int line(int d, int mode, void* psi, const void* tk, cudaStream_t st);
    int cnpass(int d, void* psi, cudaStream_t st);
    int enqueue_step(void* psi, bool first, bool last, cudaStream_t st);
    int col_capacity(int d) const;
    int set_potential(const double* U_re_im);   // host complex [nz][ny][nx]
    ~Plan3D();
};
}  // namespace soft

struct soft_plan {
    int kind = 0;              // 1: 1D (single or batch), 2: 2D, 3: 3D
    bool single = false;
    int prec = SOFT_C128;
    soft_options opt{};
    double dt = 0;
    int64_t last_launches = 0;

    // ---- 1D
    struct InstHost {
        int tab;
        int64_t off;
        int n;
        int has_field, fcls;
        double E0;
    };
    std::vector<std::unique_ptr<soft::Tables1D>> tabs;
    std::vector<InstHost> inst;
    std::vector<soft::Group1D> groups;
    // instances of the persistent kernel: descriptors in pack order, packs
    int npacks = 0;
    bool use_persist = false;      // launch the packs' sizes through the persistent kernel
    soft::Inst1D* d_pinst = nullptr;
    void* d_packs = nullptr;
    int* d_pcount = nullptr;
    std::vector<soft::Inst1D> h_obs;
    soft::Inst1D* d_inst_obs = nullptr;
    std::vector<double> h_cls;     // (omega, Tp) per pulse class
    int ncls = 0;
    double call_cls[2] = {0, 0};   // the class slot used by soft_step's field
    double* d_cls = nullptr;
    double* d_ftab = nullptr;
    int64_t ftab_cap = 0;
    int* d_status = nullptr;
    int64_t total = 0;

    // graph replay of one chunk (pulse table, size groups on parallel streams)
    static constexpr size_t MAX_SIDE = 16;
    double* d_t0 = nullptr;
    cudaStream_t side[MAX_SIDE] = {};
    cudaEvent_t ev_join[MAX_SIDE] = {};
    cudaEvent_t ev_fork = nullptr;
    bool side_ready = false;
    cudaGraphExec_t gexec = nullptr;
    void* gpsi = nullptr;
    int64_t gchunk = 0, glaunches = 0;
    cudaStream_t gstream = nullptr;

    soft::Inst1D descriptor(int i) const;
    int build_1d_device();
    int set_single_field(const soft_field* f, cudaStream_t st);
    int enqueue_chunk(void* psi, int64_t chunk, cudaStream_t st);
    int ensure_side();
    int time_schedules();
    int step_1d(void* psi, int64_t nsteps, double* t_inout, cudaStream_t st);
    soft::Sse1D* s1 = nullptr;     // stationary solver of a single 1D plan (sse1d.cu)
    soft::Surf1D* sf = nullptr;    // surface-sampling tables (soft1d_surf.cu)

    // ---- 2D (plan2d.cu), learned correction (nn.cu)
    soft::Plan2D* p2 = nullptr;
    soft::NNState* nn = nullptr;
    int step_2d(void* psi, int64_t nsteps, double* t_inout, cudaStream_t st);
    int64_t points_2d() const;
    void free_2d();

    // ---- 3D (plan3d.cu)
    soft::Plan3D* p3 = nullptr;
    int step_3d(void* psi, int64_t nsteps, double* t_inout, cudaStream_t st);
    int64_t points_3d() const;
    void free_3d();

    ~soft_plan();
};

int create_2d(const soft_grid* grid, const double* box, double R0, double theta, double dt,
              const soft_options& o, soft_plan** out);
int create_3d(const soft_grid* grid, const double* box, double R0, double theta, double dt,
              const soft_options& o, soft_plan** out);
