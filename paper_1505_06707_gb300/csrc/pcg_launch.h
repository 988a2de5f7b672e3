// Launchers of the stationary-solver kernels (pcg_kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "soft.h"

namespace soft {

struct PcgGeo;

enum { STAGE_FNORM = 0, STAGE_RHO = 1, STAGE_ALPHA = 2, STAGE_RNORM = 3, STAGE_BETA = 4, STAGE_BETA_FLEX = 5,
       STAGE_RNORM_RU = 6, STAGE_TRUE = 7 };

struct PcgState {                 // device pointers, per energy unless noted
    double2* rho;
    double2* alpha;
    double2* beta;
    double* relres;
    double* fnorm2;               // scalar
    int* active;
    int* iters;
    int* status;
    int* nactive;                 // scalar
    double tol;
    // reliable updates (A computing in FP32): relative residual at the last
    // true-residual update, the update flags, the drop that triggers one and
    // the most iterations between two; per energy the iteration of the last
    // update, the mode (bit 0: A in FP64 from now on, bit 1: restart with
    // beta = 0) and the launch masks of the FP32 and FP64 A passes
    double* rref;
    int* upd;
    double delta;
    int maxgap;
    int* lastu;
    int* mode;
    int* act32;
    int* act64;
};

// which: 0 = A row pass (a = p, b = w), 1 = preconditioner row pass 1
// (a = r, b = t), 2 = preconditioner row pass 2 (a = t, b = z, c = r for r^T z)
int pcg_row(int logn, int which, const PcgGeo& g, const void* a, void* b, const void* c,
            const double* E, const int* act, double2* part, int nE, cudaStream_t st);
// which: 0 = A column pass (a = p, b = w, partial p^T w), 1 = preconditioner
// column pass (b = t in place)
int pcg_col(int logn, int which, const PcgGeo& g, const void* a, void* b, const double* E,
            const int* act, double2* part, int nE, cudaStream_t st);
int pcg_col_blocks(int nx);
// the banded preconditioner computing in FP32: which 1 = row pass 1 (a = r,
// b = t), 2 = row pass 2 (a = t, b = z, c = r for r^T z); r and z complex128,
// t complex64; column pass on t in place
int pcg_pc32_row(int logn, int which, const PcgGeo& g, const void* a, void* b, const void* c,
                 const int* act, double2* part, int nE, cudaStream_t st);
int pcg_pc32_col(int logn, const PcgGeo& g, void* b, const double* E, const int* act, int nE,
                 cudaStream_t st);

// A on complex64 vectors (p in, w out), computing in FP32 (a32, FP32 tables)
// or in FP64 (a64f, FP64 tables): row pass (w = ...) then column pass
// (w += ..., partials of p^T w at part[e * pstride + b] for its blocks b,
// zero up to pstride >= its block count)
int pcg_a32_row(int logn, const PcgGeo& g, const void* p, void* w, const double* E, const int* act,
                int nE, cudaStream_t st);
int pcg_a32_col(int logn, const PcgGeo& g, const void* p, void* w, const int* act, double2* part,
                int pstride, int nE, cudaStream_t st);
int pcg_a64f_row(int logn, const PcgGeo& g, const void* p, void* w, const double* E, const int* act,
                 int nE, cudaStream_t st);
int pcg_a64f_col(int logn, const PcgGeo& g, const void* p, void* w, const int* act, double2* part,
                 int pstride, int nE, cudaStream_t st);
// the banded preconditioner in FP32 on complex64 vectors: which 1 = row pass
// 1 (a = r, b = t); 2 = row pass 2 (a = t, b = z; with r the partials of r^T z
// in part, with w those of z^T w in part2); column pass: pcg_pc32_col
int pcg_pc32f_row(int logn, int which, const PcgGeo& g, const void* a, void* b, const void* r, const void* w,
                  const int* act, double2* part, double2* part2, int nE, cudaStream_t st);

int vec_init(const void* f, void* x, void* r, int64_t N, int nE, cudaStream_t st);
int vec_norm2(const void* f, int64_t N, double2* part, int nparts, cudaStream_t st);
int vec_xr(void* x, void* r, const void* p, const void* w, const double2* alpha, const int* act,
           int64_t N, int nE, double2* part, int nparts, cudaStream_t st);
int vec_p(void* p, const void* z, const double2* beta, const int* act, int64_t N, int nE, int copy,
          cudaStream_t st);
// r = f - t (complex128) for the active energies
int vec_sub(const void* f, const void* t, void* r, const int* act, int64_t N, int nE, cudaStream_t st);
int pcg_scalars(int stage, int nE, const double2* part, int nparts, const PcgState& s,
                cudaStream_t st, const double2* part2 = nullptr);
// one flexible-GCR orthogonalisation of slot `slot` against the other mu-1
// stored (P, Q = A P) pairs, then alpha = <Q_s, r>/<Q_s, Q_s> (Hermitian)
int gcr_step(int phase, void* Pb, void* Q, int64_t slot_stride, int mu, int ld, int slot, double2* beta,
             double* qnorm, const void* r, const int* act, int64_t N, int nE, double2* gpart, double2* part,
             double2* part2, int nparts, const PcgState& s, cudaStream_t st);
// mixed iteration: complex64 r, p, z, w; double-float increment (xh, xl)
int vec_init32(const void* f, void* x, void* r, void* xh, void* xl, int64_t N, int nE, cudaStream_t st);
int vec_xr32(void* xh, void* xl, void* r, const void* p, const void* w, const double2* alpha, const int* act,
             int64_t N, int nE, double2* part, int nparts, cudaStream_t st);
int vec_p32(void* p, const void* z, const double2* beta, const int* act, int64_t N, int nE, int copy,
            cudaStream_t st);
int vec_fold(void* x, void* xh, void* xl, const int* mask, int64_t N, int nE, cudaStream_t st);
// r = f - t (t = A x in FP64) rounded to complex64, for the energies with
// upd set; partials of ||f - t||^2 in FP64
int vec_res32(const void* f, const void* t, void* r, const int* upd, int64_t N, int nE, double2* part,
              int nparts, cudaStream_t st);
// partials of the bilinear forms r^T z and z^T w (flexible CG)
int vec_dot2(const void* r, const void* z, const void* w, const int* act, int64_t N, int nE,
             double2* part1, double2* part2, int nparts, cudaStream_t st);

}  // namespace soft
