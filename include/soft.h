/*
 * soft.h -- C ABI of the GB300 library for the method of Serov & Sergeeva,
 * "Solution of the Schroedinger equation using exterior complex scaling and
 * fast Fourier transform" (arXiv:1505.06707).
 *
 *   - soft_create / soft_create_batch / soft_step / soft_step_batch:
 *     the exterior-complex-scaled split-operator FFT time step of Sec. II,
 *       psi(t+tau) = F^-1 e^{-iK tau/2} F e^{-iU tau/2} e^{-iC tau}
 *                    e^{-iU tau/2} F^-1 e^{-iK tau/2} F psi(t)
 *     (the scheme printed after Eq. C_FD), with e^{-iC tau} by Crank-Nicolson.
 *   - sse_pcg_solve: the stationary equation A psi = f,
 *     A = F^-1 K F + C + U - E I (Sec. III, under Eq. linsys), by
 *     complex-symmetric conjugate gradients with the FFT preconditioner of
 *     Eq. PreconFFT or the banded ECS preconditioner of Eq. PreconFFT_ECS.
 *
 * Conventions shared by every call
 *   Grid.   Axis d has n[d] = 2^m points x_j = a + h (j + 1/2), j = 0..n-1,
 *           h = (b - a)/n (Sec. II, Eq. DVRgrid, 0-based).  The box must be
 *           symmetric (a = -b): the contour q(x) is even.
 *   State.  psi holds samples psi~(x_j) of the scaled wave function
 *           psi~ = sqrt(q) psi(z(x)) (Sec. II, Eq. psi_zx), interleaved complex
 *           (re, im), float for SOFT_C64 and double for SOFT_C128.  2D states
 *           are row-major [ny][nx] (x fastest).  The paper's sqrt(h) DVR factor
 *           (Sec. II after Eq. FFTbasis) is dropped: every operator is linear.
 *   Memory. Pointers documented "device" must point to CUDA device memory of
 *           the calling thread's current device, owned by the caller and
 *           aligned to 16 bytes.  Pointers documented "host" are ordinary
 *           host memory.  Plans own their tables and workspaces.
 *   Streams. Every call that takes a cudaStream_t (passed as void*, NULL =
 *           legacy default stream) only enqueues work; results are valid once
 *           that stream has been synchronised.  A plan must not be used from
 *           two streams at once.
 *   Errors. Every call returns an int status (SOFT_OK = 0 or a negative
 *           soft_status).  No call aborts, traps or throws.  Arguments are
 *           checked on the host before any launch; device-side failures are
 *           reported through status words read back by the host.
 */
#ifndef SOFT_H
#define SOFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SOFT_OK = 0,
    SOFT_ERR_INVALID_ARG = -1,   /* NULL pointer, non-positive size, bad enum  */
    SOFT_ERR_NOT_POW2 = -2,      /* grid size not a power of two              */
    SOFT_ERR_OOM = -3,           /* cudaMalloc or a host allocation failed    */
    SOFT_ERR_CUDA = -4,          /* a CUDA runtime call failed                */
    SOFT_ERR_NOT_CONVERGED = -5, /* PCG hit maxit; outputs are still written  */
    SOFT_ERR_BREAKDOWN = -6,     /* PCG: p^T A p or r^T z vanished            */
    SOFT_ERR_TIMEOUT = -7,       /* a bounded device wait gave up             */
    SOFT_ERR_NONFINITE = -8,     /* NaN/Inf in an input or a result           */
    SOFT_ERR_UNSUPPORTED = -9,   /* size/precision combination not built      */
    SOFT_ERR_SETUP = -10,        /* plan tables failed a self-check           */
    SOFT_ERR_TOO_LARGE = -11     /* request exceeds a fixed-size scratch area  */
} soft_status;

typedef enum { SOFT_C64 = 1, SOFT_C128 = 2 } soft_prec;

/* Contour q(x) of Sec. II, Eq. ECSintdef, used on every axis.
 *   SHARP: q = 1 for |x| <= R0, e^{i theta} beyond (Sec. IV, first contour).
 *   SECS:  q = exp[i theta (|x| - R0)/(b - R0)] beyond R0: Eq. qSECS (Sec. IV)
 *          with its final angle pi/4 made the parameter theta.
 *   TFECS: q = sqrt(1 + i y~(s)), y~ = alpha[(1-s)^-2 - (1+s)^-2 - 4s],
 *          s = (|x| - R0)/(b - R0) (Sec. IV, Eq. qTFECS).
 * The comparison absorbers of Sec. IV keep the contour real (q = 1, z = x,
 * so C = 0 and no strip) and add a complex potential beyond R0 = r_s:
 *   CAP:   U_a = E_CAP [1 - q^2] with the SECS q (final angle theta),
 *          Eq. CAP_via_q;
 *   TFAP:  U_a = -i (k_min^2/2) y(s), y(s) = [a s - b s^3 + 4/(1-s)^2
 *          - 4/(1+s)^2]/c^2, a = c^3 - 16, b = c^3 - 17, c = 2.622057
 *          (Eqs. TFAP, yTFAP).
 * Plans with an absorber take no laser field (SOFT_ERR_UNSUPPORTED).      */
typedef enum {
    SOFT_CONTOUR_SHARP = 0, SOFT_CONTOUR_SECS = 1, SOFT_CONTOUR_TFECS = 2,
    SOFT_ABSORB_CAP = 3, SOFT_ABSORB_TFAP = 4
} soft_contour;

typedef struct {
    int ndim;        /* 1, 2 or 3                                          */
    int64_t n[3];    /* points per axis (x, y, z), powers of two; unused
                        entries ignored                                    */
} soft_grid;

/* Optional settings; NULL means the defaults given in brackets. */
typedef struct {
    int prec;            /* soft_prec [SOFT_C128]                            */
    int contour;         /* soft_contour [SOFT_CONTOUR_SHARP]                */
    double tfecs_alpha;  /* alpha of Eq. qTFECS [0.5]                        */
    double soft_a2;      /* a^2 of U = -Z/sqrt(z^2 + a^2), z complex [2.0]   */
    double charge;       /* Z [1.0]; 0 gives U = 0                           */
    int band_width;      /* N_BW of the banded preconditioner [10]           */
    int autotune;        /* 1: time the built kernel variants of every 1D size
                            at plan creation and keep the fastest [0]       */
    double cap_energy;   /* E_CAP of the linear CAP [2.0]                    */
    double tfap_kmin;    /* k_min of TFAP [0.25]                             */
    int persistent;      /* batch plans: 1 advances the instances with
                            N = 2048 .. 16384 by one persistent kernel that
                            takes packs of same-size instances from a queue,
                            largest N first; 0 launches one kernel per size
                            group.  With autotune the plan times both on one
                            16-step chunk and keeps the faster [1]           */
} soft_options;

/* Laser pulse (length gauge, x-polarised), E(t) = E0 sin^2(pi t/T) sin(omega t)
 * for 0 <= t <= T = ncycles 2 pi/omega, zero outside.  It couples as
 * U_L = E(t) xc with xc = clamp(x, -R0, R0): the field is held constant
 * inside the scaled strips (continuing E z into complex z would grow
 * exponentially there).  U is taken at t + tau/2 (Sec. II under Eq. SSFFT). */
typedef struct {
    double E0, omega, ncycles;
} soft_field;

typedef struct soft_plan soft_plan;   /* opaque, library-owned */

void soft_default_options(soft_options* opt);

/* soft_create -- build the tables of one problem (Sec. II, Sec. III).
 *   grid   host; 1D, 2D or 3D sizes.  2D grids are stored [ny][nx], 3D
 *          grids [nz][ny][nx] (x fastest).  2D axes take 256 .. 2048
 *          points, 3D axes 64 .. 2048.
 *   box    host; a0, b0 [, a1, b1 [, a2, b2]] with a = -b on each axis.
 *   R0     onset |x| of the scaling, 0 < R0 < b on each axis.
 *   theta  rotation angle of the sharp contour, final angle of SECS (pi/4 is
 *          the paper's SECS); ignored by TFECS.
 *   dt     time step tau (may be negative: backwards propagation).
 *   opt    host, may be NULL.
 *   out    host; receives the plan.
 * Tables are computed on the host in FP64 and uploaded once.  Fails with
 * SOFT_ERR_NOT_POW2 for sizes that are not powers of two in [64, 16384],
 * SOFT_ERR_SETUP if the strip Crank-Nicolson factorisation is not accurate
 * to 1e-12 in FP64.  With opt->autotune the plan times every built
 * (elements per thread, radix) variant of each 1D size on the device and keeps
 * the fastest; this launches kernels and allocates temporary buffers. */
int soft_create(const soft_grid* grid, const double* box, double R0, double theta,
                double dt, const soft_options* opt, soft_plan** out);

/* soft_create_batch -- `count` independent 1D problems that advance together
 * (one launch for all).  grids[count], boxes[2*count], R0[count],
 * theta[count] and fields[count] (NULL = no field) are host arrays.  The
 * states are packed back to back in creation order; soft_batch_layout gives
 * the element offset of each. */
int soft_create_batch(int count, const soft_grid* grids, const double* boxes,
                      const double* R0, const double* theta, const soft_field* fields,
                      double dt, const soft_options* opt, soft_plan** out);

/* offsets: host int64[count]; element (not byte) offset of each instance in
 * the packed state.  total: host; total number of complex elements. */
int soft_batch_layout(const soft_plan* plan, int64_t* offsets, int64_t* total);

/* soft_step -- advance psi by nsteps steps of the scheme printed after
 * Eq. C_FD (Sec. II).  psi: device, in/out.  field: host, may be NULL (batch
 * plans use their own per-instance fields and ignore it).  t_inout: host,
 * the time at entry, advanced by nsteps*dt on return.  The half-kinetic
 * factors of consecutive steps inside one call are merged (the scheme is
 * unchanged up to rounding).  nsteps = 0 is a no-op.  2D and 3D plans take
 * no field (it is ignored) and run their steps as passes over the grid's
 * lines (rows, then columns), with C = C_x + C_y (+ C_z) as Kronecker sums
 * so that e^{-iC tau} factors into one CN per axis; the middle steps are
 * replayed from a CUDA graph captured on the first call with a given state
 * pointer and stream. */
int soft_step(soft_plan* plan, void* psi, int64_t nsteps, const soft_field* field,
              double* t_inout, void* stream);

/* soft_step_batch -- soft_step for a batch plan; psi is the packed state.
 * Calls are replayed from a CUDA graph (captured on the first call with a
 * given state pointer, stream and step count): the pulse-shape table, the
 * persistent kernel over the instances with N = 2048 .. 16384 (one CTA per
 * SM; 1, 2, 2, 4 instances of N = 16384, 8192, 4096, 2048 per work item
 * for complex64, 1, 1, 2, 2 for complex128) and one kernel per remaining
 * size group, on parallel branches so that their CTAs share the GPU. */
int soft_step_batch(soft_plan* plan, void* psi, int64_t nsteps, double* t_inout,
                    void* stream);

/* soft_observe -- norm inside the unscaled region, h sum_{|x_j|<R0} |psi_j|^2,
 * and the probability flux j = Im(psi^* dpsi/dx) at x = -R0 and x = +R0
 * (two-point mean and difference across the edge, which lies half-way
 * between grid points).  These are the quantities a t-SURFF analysis draws
 * from the propagated state (Sec. I, Sec. IV).  1D plans only.
 *   psi       device (packed state for batch plans).
 *   norm_in   device double[count].
 *   flux      device double[2*count] (left, right per instance).
 * FP64 accumulation. */
int soft_observe(const soft_plan* plan, const void* psi, double* norm_in, double* flux,
                 void* stream);

/* soft_step_status -- wait for the work queued on `stream` and report whether
 * a step of this 1D plan (single or batch) has left a non-finite value in a
 * state since the last query: each step kernel tests its instance's first
 * element after its last step, where a NaN or Inf anywhere in the state has
 * arrived through the FFT.  Returns SOFT_ERR_NONFINITE and clears the flag if
 * so, SOFT_OK otherwise; SOFT_ERR_UNSUPPORTED for 2D plans.  The step calls
 * themselves never wait for the device, so they cannot report it. */
int soft_step_status(soft_plan* plan, void* stream);

/* soft_step_surface -- soft_step on a single 1D complex128 plan (N = 256 ..
 * 8192) that also samples the wave function at the two boundaries
 * x = +R0 and x = -R0 of the unscaled region after every step: the
 * quantities the amplitude extraction of the paper's test draws from the
 * propagation (t-SURFF part of t&E-SURFF, Sec. I and Sec. IV).  psi and
 * dpsi/dx there are those of the trigonometric interpolant of the grid
 * function (the FFT representation of Sec. II), taken from the spectrum
 * inside the step kernel.
 *   samples  device complex128 [nsteps + 1][4]: psi(R0), psi'(R0), psi(-R0),
 *            psi'(-R0) at t_inout + s dt, s = 0 .. nsteps.
 * Other arguments as soft_step.  SOFT_ERR_UNSUPPORTED for other plans. */
int soft_step_surface(soft_plan* plan, void* psi, int64_t nsteps, const soft_field* field,
                      double* t_inout, void* samples, void* stream);

/* sse_surff -- momentum amplitudes by t&E-SURFF (Sec. I, Sec. IV) for a
 * packet that is free beyond R0, for nE energies at once: with
 * k = sqrt(2 E) and T = t0 + (nsamples - 1) dt,
 *   A(+-k) = -+ (i/2) (2 pi)^-1/2 e^{-+ik R0} [ int_t0^T e^{iEt} g(t) dt
 *            + i e^{iET} (phi' +- ik phi)(+-R0) ],   g = psi' +- ik psi at +-R0,
 * where (E - H) phi = psi(T): the flux through the boundary up to T
 * (t-SURFF) plus the rest of the packet through the stationary equation
 * with right-hand side psi(T) (E-SURFF, the SSE of Sec. III).
 *   E        host double[nE], E > 0.
 *   phi      device complex128 [nE][N]: the solutions of A phi_A = psi(T)
 *            that sse_pcg_solve returns (A = H - E, so phi = -phi_A).
 *   samples  device, from soft_step_surface: nsamples rows, nsamples - 1
 *            even; the first at time t0.
 *   rule     0: Simpson's rule; 1: Filon-Simpson (e^{iEt} times the
 *            quadratic interpolant of g on each pair of steps, exact in
 *            the exponential; Sec. IV recommends it for large |k|).
 *   amp      device complex128 [nE][2]: A(+k), A(-k).
 * Single 1D complex128 plans (N = 256 .. 8192). */
int sse_surff(soft_plan* plan, int nE, const double* E, const void* phi, const void* samples,
              int64_t nsamples, double t0, int rule, void* amp, void* stream);

/* soft_set_potential -- replace the static potential of a single 1D plan,
 * a 2D plan or a 3D plan.  It enters the step as e^{-iU tau/2} (Sec. II, the
 * scheme after Eq. C_FD) and A as U - E (Sec. III, Eq. linsys); the default
 * is the soft-Coulomb potential of soft_options.
 *   U_re_im  host double[2n], interleaved complex: U at the complex-scaled
 *            grid points z(x_i) (2D: [ny][nx], 3D: [nz][ny][nx], x fastest).
 *            The plan's comparison-absorber potential (CAP / TFAP contours)
 *            is added.
 *   n        grid points (N, nx * ny or nx * ny * nz).
 * The plan's potential tables (and the stationary solver's, once built) are
 * rewritten in place after a device synchronisation, so call it between
 * steps; captured graphs stay valid.  SOFT_ERR_UNSUPPORTED for batch plans,
 * SOFT_ERR_INVALID_ARG for a size mismatch, SOFT_ERR_NONFINITE for a
 * non-finite value. */
int soft_set_potential(soft_plan* plan, const double* U_re_im, int64_t n);

/* sse_pcg_solve -- solve A psi_e = f for nE energies E[e] by complex-symmetric
 * CG (Sec. III: the unconjugated form r^T z replaces the inner product),
 * x0 = 0, stopping when ||r||_2 / ||f||_2 < tol (Hermitian norms, FP64).
 * On 2D plans with precond 0, 1 and 4 the stopping residual is the true
 * one: each energy that converged on the recursive residual restarts from
 * its x with r = f - A x and retires after at least one more iteration
 * (iters counts it); precond 5 decides on the true FP64 residual anyway.
 * 1D plans (single instance, N = 256 .. 2048, complex128) take precond 0
 * and 1: one CTA per energy runs the whole iteration with its vectors in
 * shared memory (one launch for all energies); 2D plans take every mode.
 *   E        host double[nE].
 *   rhs      device, one right-hand side f shared by all energies.
 *   psi_out  device, nE consecutive solutions.
 *   precond  0: simple FFT preconditioner (Eq. PreconFFT);
 *            1: banded ECS preconditioner (Eq. PreconFFT_ECS);
 *            2: the banded preconditioner plus the plan's learned correction
 *               z <- z + s NN(z/s), s = RMS of z per energy, inside flexible
 *               GCR with the last 16 directions (minimal residual with
 *               Hermitian inner products: valid for a preconditioner that
 *               changes between iterations); grids with nx % 128 == 0;
 *            3: the banded preconditioner alone inside the same flexible GCR
 *               (the reference for what the learned correction gains);
 *            4: the banded preconditioner computing in FP32 (its FFTs, band
 *               products and tables; r in and z out stay complex128, and
 *               A, the residual and the dots stay FP64), in COCG with the
 *               flexible beta = z'^T (r' - r) / r^T z (FP32 rounding leaves
 *               the preconditioner not exactly symmetric);
 *            5: mixed precision: A and the banded preconditioner compute
 *               in FP32 on complex64 r, p, z, w inside the iteration (FP32
 *               products, FP64 sums for the dots); the solution increment
 *               accumulates in double-float.  Reliable updates: once the
 *               recursive residual has dropped tenfold since the last
 *               update (or below tol, or after 200 iterations), the
 *               increment is folded into the complex128 psi and the
 *               residual replaced by the true f - A psi with A in FP64;
 *               only that true residual decides convergence, so the
 *               stopping test means the same as for 0-4.  An energy whose
 *               true residual has not halved between two updates
 *               continues with the FP64 A, after a restart; if it stalls
 *               again, it is finished by the all-FP64 COCG of precond 1
 *               started from its current psi (up to maxit more
 *               iterations).  iters_out counts all iterations.
 *   iters_out, relres_out: host int[nE], double[nE]; may be NULL.
 * Returns SOFT_ERR_NOT_CONVERGED if any energy stopped at maxit (its last
 * iterate is written), SOFT_ERR_BREAKDOWN on a vanishing CG denominator.
 * Workspace (and, for precond 2/3, 32 direction vectors per energy) is
 * allocated by the plan on first use.  C128 plans only. */
int sse_pcg_solve(soft_plan* plan, const double* E, int nE, const void* rhs, void* psi_out,
                  double tol, int maxit, int precond, int* iters_out, double* relres_out,
                  void* stream);

/* sse_apply_A / sse_apply_A32 / sse_apply_precond -- one application of A
 * (Sec. III under Eq. linsys) or of the chosen preconditioner, for one
 * energy, device in and out (x and y must not alias); 1D plans take
 * sse_apply_A and precond 0 and 1 (SOFT_ERR_UNSUPPORTED otherwise).  sse_apply_A32
 * computes A in FP32 on complex64 x and y, as precond 5 does inside its
 * iteration; the others take complex128.  Exposed for testing and for
 * callers that run their own Krylov method; precond 0, 1 or 4 (as in
 * sse_pcg_solve). */
int sse_apply_A(soft_plan* plan, double E, const void* x, void* y, void* stream);
int sse_apply_A32(soft_plan* plan, double E, const void* x, void* y, void* stream);
int sse_apply_precond(soft_plan* plan, double E, int precond, const void* x, void* y,
                      void* stream);

/* soft_step_noalloc -- soft_step for a single-instance 1D plan that allocates
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine.  The
 * paper has no counterpart; this exists for callers that cannot allocate
 * device memory while stepping (real-time loops where an allocation could
 * stall, hosts whose device memory is owned by an external manager,
 * embeddings that forbid allocation after start-up).  Its scratch (pulse
 * table, descriptor, status word) is one file-scope device array of about
 * 130 KB that every GPU loading the library keeps until exit.
 *   psi, field, t_inout, stream: as soft_step.
 *   nsteps: at most 16384 per call; larger requests return SOFT_ERR_TOO_LARGE
 *           without touching psi.
 * All calls share the array and it keeps the last call's contents; each call
 * rewrites what it uses and clears the status word first.  Calls that overlap
 * on the GPU race on the array: serialise them.  The first call on a device
 * looks up the array's device address with that device current; make it
 * before any stream capture. */
int soft_step_noalloc(const soft_plan* plan, void* psi, int64_t nsteps, const soft_field* field,
                      double* t_inout, void* stream);

/* Learned correction of the FFT preconditioner.  The paper has no learned
 * component; the network only corrects the output of Eq. PreconFFT_ECS inside
 * a flexible CG, and the plain preconditioner stays available (precond 1).
 * Network: 3x3 convolutions 2 -> 32 -> 32 -> 2 channels (real and imaginary
 * parts), ReLU between layers, periodic padding, BF16 weights and
 * activations with FP32 accumulation on the tensor cores.  The 10434 FP32
 * parameters are, in order: W1[32][2][3][3], b1[32], W2[32][32][3][3], b2[32],
 * W3[2][32][3][3], b3[2] (out[o](y,x) = b[o] + sum W[o][i][dy+1][dx+1]
 * in[i](y+dy, x+dx), indices mod H, W).  Every 2D plan owns one network,
 * initialised from a fixed seed on first use.
 *   Fields: device complex64 arrays [n][H][W], W a multiple of 128, H >= 3,
 *   at most 65535 fields per call (SOFT_ERR_TOO_LARGE beyond; for the
 *   solver's learned modes, at most 65535 energies).
 * sse_nn_set_weights / sse_nn_get_weights: host float[10434].
 * sse_nn_forward: out = NN(x), device float [n][H][W][2].
 * sse_nn_grad: mean-square loss of NN(x) against targets and its gradient
 *   (host float[10434]); no update.
 * sse_nn_train: `steps` Adam steps (lr, beta 0.9/0.999) on minibatches of
 *   `batch` fields drawn from the n inputs with the seed; loss_out: host
 *   double[steps] or NULL.
 * The convolutions with 32 input channels run on tcgen05 with a bounded
 * completion wait; if one runs out, its outputs are NaN and sse_nn_grad /
 * sse_nn_train return SOFT_ERR_TIMEOUT (sse_nn_forward and the solver's
 * correction show it as non-finite values). */
int sse_nn_set_weights(soft_plan* plan, const float* w);
int sse_nn_get_weights(soft_plan* plan, float* w);
int sse_nn_forward(soft_plan* plan, const void* x, int n, int H, int W, void* out, void* stream);
int sse_nn_grad(soft_plan* plan, const void* inputs, const void* targets, int n, int H, int W,
                float* grad_out, double* loss_out, void* stream);
int sse_nn_train(soft_plan* plan, const void* inputs, const void* targets, int n, int H, int W,
                 int steps, int batch, double lr, uint64_t seed, double* loss_out, void* stream);

void soft_destroy(soft_plan* plan);
const char* soft_strerror(int status);

/* Plan queries: number of instances, grid points of instance i, the element
 * precision, and the number of kernel launches the last call enqueued. */
int soft_plan_count(const soft_plan* plan);
int64_t soft_plan_points(const soft_plan* plan, int i);
int soft_plan_prec(const soft_plan* plan);
int64_t soft_last_launches(const soft_plan* plan);

#ifdef __cplusplus
}
#endif
#endif /* SOFT_H */
