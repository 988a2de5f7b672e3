// soft_step_noalloc: the single-instance 1D step for callers that must not
// allocate device memory while stepping.
//
// Who needs it: code that advances a wave function from a context where
// cudaMalloc is off limits -- a real-time or latency-bounded loop where an
// allocation could stall or fail, a host thread that runs under an external
// memory manager that owns every device allocation, or an embedding that
// forbids allocation after start-up.  soft_step itself allocates nothing per
// call either, but it relies on scratch (the per-call pulse table and the
// status word) that the plan allocated with cudaMalloc; this entry point
// instead takes that scratch from one fixed, file-scope device array.
//
// Limits and sharing:
//   - the array holds at most NOALLOC_MAX_STEPS pulse values, so one call
//     accepts at most that many steps (SOFT_ERR_TOO_LARGE beyond it);
//   - every GPU that loads the library keeps the array (about 130 KB) until
//     the process exits;
//   - all calls share the array and it keeps the last call's contents: each
//     call rewrites what it reads (descriptor, pulse table) and clears the
//     status word first.  Calls whose work overlaps on the GPU (other streams,
//     other host threads) race on it and must be serialised by the caller;
//   - the first call on a device looks up the array's device address with
//     that device current (once per device); make that first call before any
//     stream capture.
#include <mutex>

#include "plan_internal.h"

namespace {

constexpr int64_t NOALLOC_MAX_STEPS = 16384;

struct NoallocScratch {
    soft::Inst1D desc;                 // descriptor of the one instance
    double cls[2];                     // omega, pulse length
    int status;
    int pad[3];
    double pulse[NOALLOC_MAX_STEPS];   // pulse shape at each step's midpoint
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
NoallocScratch* g_addr[MAX_DEVICES] = {nullptr};

int scratch_address(NoallocScratch** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SOFT_ERR_CUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return SOFT_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        // host code must not use &g_noalloc_scratch directly: it names a host
        // stand-in, not the device copy
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SOFT_ERR_CUDA;
        g_addr[dev] = static_cast<NoallocScratch*>(p);
    }
    *out = g_addr[dev];
    return SOFT_OK;
}

// Writes this call's descriptor and pulse class into the scratch and clears
// its status word.  The values travel as kernel arguments, so no host buffer
// has to outlive the call.
__global__ void noalloc_setup_kernel(NoallocScratch* sc, soft::Inst1D desc, double omega, double Tp) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        sc->desc = desc;
        sc->cls[0] = omega;
        sc->cls[1] = Tp;
        sc->status = 0;
    }
}

}  // namespace

extern "C" int soft_step_noalloc(const soft_plan* P, void* psi, int64_t nsteps,
                                 const soft_field* field, double* t_inout, void* stream) {
    if (!P || !psi || !t_inout || nsteps < 0) return SOFT_ERR_INVALID_ARG;
    if (P->kind != 1 || !P->single || P->groups.size() != 1) return SOFT_ERR_INVALID_ARG;
    if (nsteps > NOALLOC_MAX_STEPS) return SOFT_ERR_TOO_LARGE;
    if (nsteps == 0) return SOFT_OK;
    NoallocScratch* sc = nullptr;
    int rc = scratch_address(&sc);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    // descriptor of the instance with this call's field (pulse class 0 of the scratch)
    soft::Inst1D d = P->descriptor(0);
    double cls[2] = {1.0, 1.0};
    d.has_field = 0; d.fcls = 0; d.E0 = 0.0;
    if (field && field->E0 != 0.0) {
        if (!(field->omega > 0 && field->ncycles > 0)) return SOFT_ERR_INVALID_ARG;
        if (P->opt.contour >= SOFT_ABSORB_CAP) return SOFT_ERR_UNSUPPORTED;   // absorbers: no field
        cls[0] = field->omega;
        cls[1] = field->ncycles * 2 * 3.14159265358979323846 / field->omega;
        d.has_field = 1;
        d.E0 = field->E0;
    }
    noalloc_setup_kernel<<<1, 32, 0, st>>>(sc, d, cls[0], cls[1]);
    if ((rc = soft::cuda_status(cudaGetLastError()))) return rc;
    if (d.has_field) {
        rc = soft::launch_field_table(sc->cls, 1, *t_inout, P->dt, nsteps, sc->pulse,
                                      NOALLOC_MAX_STEPS, st);
        if (rc) return rc;
    }
    const soft::Group1D& g = P->groups[0];
    rc = soft::launch_soft1d(P->prec, g.logn, g.loge, g.logrm, &sc->desc, 1, psi, nsteps,
                             sc->pulse, NOALLOC_MAX_STEPS, &sc->status, st, nullptr);
    if (rc) return rc;
    *t_inout += (double)nsteps * P->dt;
    return SOFT_OK;
}
