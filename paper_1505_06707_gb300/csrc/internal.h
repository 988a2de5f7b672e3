// Internal declarations shared by the host plan code and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <memory>
#include <string>
#include <vector>

#include "soft.h"
#include "host_tables.h"

namespace soft {

using cd = std::complex<double>;

// Device descriptor of one 1D instance (read by the 1D step kernel).
struct Inst1D {
    int64_t off;          // element offset of the instance in the packed state
    const void* TK;       // e^{-i k^2 tau/2}/N, forward FFT output order, last-pass transposed
    const void* TKh;      // e^{-i k^2 tau/4}/N, same order (first/last half step)
    const void* TV;       // e^{-iU0 tau} off the strip block, e^{-iU0 tau/2} on it (minus 1 for complex64)
    const void* W;        // per-pass twiddle bases (see soft1d.cuh)
    const void* cn;       // strip CN coefficients, chunk-transposed (soft1d.cuh, strip_cn_1d)
    const void* TVs;      // TV on the strip rows, same transposed order
    int nb;               // strip block length (0: no absorbing term)
    int blk0;             // first grid index of the block (cyclic)
    double x0, h, R0, tau;
    double E0;            // field amplitude; the pulse shape comes from a per-call table
    int has_field;
    int fcls;             // index of the pulse-shape class in that table
    int iL, iR;           // x_n <= -R0 for n < iL, x_n >= R0 for n >= iR
    int n;                // grid points
    int pad_;
};

// Table set of one distinct 1D problem (shared by identical instances).
struct Tables1D {
    int prec = 0, logn = 0, loge = 0, logrm = 0;
    int nb = 0, blk0 = 0, iL = 0, iR = 0;
    double R0 = 0, theta = 0;
    Axis1D ax;                    // host FP64 grid, contour, C
    std::vector<cd> U0;           // potential at z(x_j)
    std::vector<cd> Uabs;         // its comparison-absorber part (zero for the ECS contours)
    void* TK = nullptr;           // device buffers in the plan's precision
    void* TKh = nullptr;
    void* TV = nullptr;
    void* W = nullptr;
    void* cn = nullptr;
    void* TVs = nullptr;
};

// Complex128 1D step plans store every pass twiddle W^{M off} for passes of
// stride up to this (the bases above it), see soft1d.cuh.
constexpr int TWFULL_MAXS = 256;

// Work item of the persistent batch kernel: up to G instances of one size.
struct Pack1D {
    int var;      // variant index in the kernel's list
    int first;    // first descriptor of the pack (descriptors in pack order)
    int count;    // instances in the pack (<= the variant's group count)
    int pad_;
};

struct Group1D {                  // instances sharing one kernel configuration
    int logn = 0, loge = 0, logrm = 0;
    bool in_persist = false;      // also in the persistent kernel's packs
    std::vector<int> members;     // instance indices
    Inst1D* d_inst = nullptr;     // device descriptors
};

// kernel launchers (defined in soft1d_*.cu)
int launch_soft1d(int prec, int logn, int loge, int logrm, const Inst1D* d_inst, int count,
                  void* psi, int64_t nsteps, const double* ftab, int64_t ftab_stride, int* d_status,
                  cudaStream_t st, size_t* smem_out);
// f_c(s) = sin^2(pi t/Tp) sin(omega t) at t = t0 + (s + 1/2) tau for each pulse class c
int launch_field_table(const double* d_cls /*omega, Tp pairs*/, int ncls, double t0, double tau,
                       int64_t nsteps, double* out, int64_t stride, cudaStream_t st);
int launch_field_table_dev(const double* d_cls, int ncls, const double* d_t0, double tau,
                           int64_t nsteps, double* out, int64_t stride, cudaStream_t st);
int soft1d_variants(int prec, int logn, int* loge, int* logrm, int maxv);
// the persistent mixed-size kernel (soft1d_persist_*.cu); packs point to
// Pack1D records, counter to the queue position (zero before the launch)
int launch_persist(int prec, const void* packs, int npacks, int* counter, const Inst1D* insts, void* psi,
                   int64_t nsteps, const double* ftab, int64_t fstride, int* status, cudaStream_t st,
                   int* ctas_out);
int persist_config(int prec, int logn, int* loge, int* logrm, int* groups);
int launch_advance_time(double* d_t, double dt, cudaStream_t st);
bool soft1d_supported(int prec, int logn, int loge, int logrm);
void soft1d_default_cfg(int prec, int logn, int* loge, int* logrm);

int launch_observe1d(int prec, const Inst1D* d_inst, int count, const void* psi,
                     double* norm_in, double* flux, cudaStream_t st);

}  // namespace soft
