/*
 * Oracle: plain FP64 CPU statement of the ECS split-operator FFT time step
 * (Serov & Sergeeva, arXiv:1505.06707, Sec. II) for 1D, 2D and 3D grids.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark load this library; the GPU library never
 * does, and the two share no code.
 *
 * Deliberate plainness:
 *   - the FFT is an iterative radix-2 transform whose twiddles are taken from
 *     libm cos/sin for every butterfly (no tables, no recurrences);
 *   - each time step is written exactly as the scheme printed under Eq. C_FD
 *     in Sec. II: four FFTs per step, the half-kinetic factor e^{-iK tau/2} on
 *     both sides (no merging across steps), e^{-iU tau/2} on both sides of
 *     e^{-iC tau};
 *   - e^{-iC tau} is the Crank-Nicolson form (1 + i tau C/2)^{-1}
 *     (1 - i tau C/2) (Sec. II, under Eq. C_FD) applied to the FULL periodic
 *     tridiagonal C of length N, solved by Sherman-Morrison on top of a
 *     tridiagonal elimination with partial pivoting; no strip restriction.
 * OpenMP only runs independent instances (or rows / columns) side by side.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ---------------------------------------------------------------- FFT --- */
/* In-place radix-2 DFT, a[m] <- sum_j a[j] exp(sign * 2 pi i m j / n),
 * unnormalised.  n must be a power of two. */
void orc_fft(cplx *a, int n, int sign)
{
    /* bit reversal permutation */
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int i = 0; i < n; i += len) {
            for (int j = 0; j < half; ++j) {
                double ang = sign * 2.0 * M_PI * (double)j / (double)len;
                cplx w = cos(ang) + I * sin(ang);
                cplx u = a[i + j], v = a[i + j + half] * w;
                a[i + j] = u + v;
                a[i + j + half] = u - v;
            }
        }
    }
}

/* ------------------------------------------------- tridiagonal solves --- */
/* Non-periodic tridiagonal solve with partial pivoting (row interchanges).
 * dl[i] = A[i+1][i], d[i] = A[i][i], du[i] = A[i][i+1]; all are copied, b is
 * overwritten by the solution.  Returns 0, or -1 on an exactly singular
 * pivot. */
static int tri_solve_pivot(int n, const cplx *dl0, const cplx *d0, const cplx *du0,
                           cplx *b, cplx *work)
{
    cplx *dl = work, *d = work + n, *du = work + 2 * n, *du2 = work + 3 * n;
    memcpy(dl, dl0, sizeof(cplx) * (n - 1));
    memcpy(d, d0, sizeof(cplx) * n);
    memcpy(du, du0, sizeof(cplx) * (n - 1));
    for (int i = 0; i < n; ++i) du2[i] = 0;
    for (int i = 0; i < n - 1; ++i) {
        if (cabs(d[i]) >= cabs(dl[i])) {           /* keep row i as pivot */
            if (d[i] == 0) return -1;
            cplx f = dl[i] / d[i];
            d[i + 1] -= f * du[i];
            b[i + 1] -= f * b[i];
        } else {                                   /* swap rows i and i+1 */
            cplx f = d[i] / dl[i];
            cplx di1 = d[i + 1];
            cplx dui1 = (i < n - 2) ? du[i + 1] : 0;
            d[i] = dl[i];
            cplx old_du = du[i];
            du[i] = di1;
            du2[i] = dui1;
            d[i + 1] = old_du - f * di1;
            if (i < n - 2) du[i + 1] = -f * dui1;
            cplx bi = b[i];
            b[i] = b[i + 1];
            b[i + 1] = bi - f * b[i + 1];
        }
    }
    if (d[n - 1] == 0) return -1;
    b[n - 1] /= d[n - 1];
    if (n > 1) b[n - 2] = (b[n - 2] - du[n - 2] * b[n - 1]) / d[n - 2];
    for (int i = n - 3; i >= 0; --i)
        b[i] = (b[i] - du[i] * b[i + 1] - du2[i] * b[i + 2]) / d[i];
    return 0;
}

/* Periodic tridiagonal solve A x = r.  sub[i] = A[i][i-1], diag[i] = A[i][i],
 * sup[i] = A[i][i+1], indices mod n.  Sherman-Morrison: A = T + u v^T with
 * u = (g,0..0,alpha), v = (1,0..0,beta/g), alpha = A[n-1][0], beta = A[0][n-1]. */
int orc_cyclic_solve(int n, const cplx *sub, const cplx *diag, const cplx *sup,
                     cplx *x, cplx *work)
{
    cplx *dl = work, *d = work + n, *du = work + 2 * n;
    cplx *y = work + 3 * n, *zz = work + 4 * n, *tw = work + 5 * n;
    cplx alpha = sup[n - 1], beta = sub[0];
    for (int i = 0; i < n - 1; ++i) { dl[i] = sub[i + 1]; du[i] = sup[i]; }
    for (int i = 0; i < n; ++i) d[i] = diag[i];
    if (alpha == 0 && beta == 0) {
        return tri_solve_pivot(n, dl, d, du, x, tw);
    }
    cplx g = (d[0] != 0) ? -d[0] : -1.0;
    d[0] -= g;
    d[n - 1] -= alpha * beta / g;
    memcpy(y, x, sizeof(cplx) * n);
    for (int i = 0; i < n; ++i) zz[i] = 0;
    zz[0] = g; zz[n - 1] = alpha;
    if (tri_solve_pivot(n, dl, d, du, y, tw)) return -1;
    if (tri_solve_pivot(n, dl, d, du, zz, tw)) return -1;
    cplx vy = y[0] + (beta / g) * y[n - 1];
    cplx vz = zz[0] + (beta / g) * zz[n - 1];
    cplx fac = vy / (1.0 + vz);
    for (int i = 0; i < n; ++i) x[i] = y[i] - fac * zz[i];
    return 0;
}

/* Crank-Nicolson factor of Sec. II: x <- (1 + i tau C/2)^{-1} (1 - i tau C/2) x
 * on the full periodic tridiagonal C. */
static int cn_apply(int n, const cplx *Cs, const cplx *Cd, const cplx *Cu,
                    double tau, cplx *x, cplx *work)
{
    cplx *rhs = work, *ms = work + n, *md = work + 2 * n, *mu = work + 3 * n;
    cplx *tw = work + 4 * n;
    cplx ih = I * tau * 0.5;
    for (int i = 0; i < n; ++i) {
        int im = (i + n - 1) % n, ip = (i + 1) % n;
        rhs[i] = x[i] - ih * (Cs[i] * x[im] + Cd[i] * x[i] + Cu[i] * x[ip]);
        ms[i] = ih * Cs[i];
        md[i] = 1.0 + ih * Cd[i];
        mu[i] = ih * Cu[i];
    }
    if (orc_cyclic_solve(n, ms, md, mu, rhs, tw)) return -1;
    memcpy(x, rhs, sizeof(cplx) * n);
    return 0;
}

/* Laser pulse E(t) = E0 sin^2(pi t/T) sin(omega t) on [0, T], T = ncyc 2pi/omega. */
static double pulse(double t, double E0, double omega, double ncyc)
{
    double T = ncyc * 2.0 * M_PI / omega;
    if (!(t >= 0.0 && t <= T)) return 0.0;
    double s = sin(M_PI * t / T);
    return E0 * s * s * sin(omega * t);
}

static void kinetic_half(cplx *psi, int n, const double *k, double tau)
{
    orc_fft(psi, n, -1);
    for (int m = 0; m < n; ++m) {
        double ph = -0.5 * k[m] * k[m] * tau * 0.5;      /* e^{-i (k^2/2) tau/2} */
        psi[m] *= (cos(ph) + I * sin(ph)) / (double)n;
    }
    orc_fft(psi, n, +1);
}

/* One instance, nsteps steps of Sec. II's ECS scheme:
 *   psi <- F^-1 e^{-iK tau/2} F e^{-iU tau/2} e^{-iC tau} e^{-iU tau/2} F^-1 e^{-iK tau/2} F psi,
 * with U(x, t + tau/2) = U0(z(x)) + E(t + tau/2) xc(x) (Sec. II under Eq. SSFFT).
 * Returns 0, or -1 on a singular CN matrix. */
int orc_step1d(int n, long nsteps, cplx *psi, const double *k, const cplx *U0,
               const double *xc, const cplx *Cs, const cplx *Cd, const cplx *Cu,
               double tau, double t0, int has_field, double E0, double omega,
               double ncyc)
{
    cplx *work = (cplx *)malloc(sizeof(cplx) * 16 * n);
    cplx *vh = (cplx *)malloc(sizeof(cplx) * n);
    if (!work || !vh) { free(work); free(vh); return -2; }
    int rc = 0;
    for (long s = 0; s < nsteps && rc == 0; ++s) {
        /* step s starts at t0 + s tau; its potential is taken at the midpoint
         * (computed directly: a running sum t += tau would drift by ~1e-10
         * over 1e4 steps) */
        double Ef = has_field ? pulse(t0 + ((double)s + 0.5) * tau, E0, omega, ncyc) : 0.0;
        for (int i = 0; i < n; ++i) {
            cplx U = U0[i] + Ef * xc[i];
            vh[i] = cexp(-I * U * tau * 0.5);
        }
        kinetic_half(psi, n, k, tau);
        for (int i = 0; i < n; ++i) psi[i] *= vh[i];
        rc = cn_apply(n, Cs, Cd, Cu, tau, psi, work);
        for (int i = 0; i < n; ++i) psi[i] *= vh[i];
        kinetic_half(psi, n, k, tau);
    }
    free(work); free(vh);
    return rc;
}

/* Independent instances side by side (OpenMP over instances).  Instance j
 * owns psi[off[j] .. off[j]+n[j]) and likewise for the per-point tables. */
int orc_step1d_batch(int count, const int *n, const long *off, long nsteps, cplx *psi,
                     const double *k, const cplx *U0, const double *xc,
                     const cplx *Cs, const cplx *Cd, const cplx *Cu,
                     const double *tau, const double *t0, const int *has_field,
                     const double *E0, const double *omega, const double *ncyc)
{
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 1) reduction(|:bad)
    for (int j = 0; j < count; ++j) {
        long o = off[j];
        int r = orc_step1d(n[j], nsteps, psi + o, k + o, U0 + o, xc + o, Cs + o, Cd + o,
                           Cu + o, tau[j], t0[j], has_field[j], E0[j], omega[j], ncyc[j]);
        if (r) bad = 1;
    }
    return bad ? -1 : 0;
}

/* --------------------------------------------------------------- 2D --- */
/* psi is [ny][nx], x fastest. */
static void fft2(cplx *psi, int nx, int ny, int sign)
{
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) orc_fft(psi + (long)y * nx, nx, sign);
    #pragma omp parallel
    {
        cplx *col = (cplx *)malloc(sizeof(cplx) * ny);
        #pragma omp for schedule(static)
        for (int x = 0; x < nx; ++x) {
            for (int y = 0; y < ny; ++y) col[y] = psi[(long)y * nx + x];
            orc_fft(col, ny, sign);
            for (int y = 0; y < ny; ++y) psi[(long)y * nx + x] = col[y];
        }
        free(col);
    }
}

static void kinetic_half2(cplx *psi, int nx, int ny, const double *kx, const double *ky,
                          double tau)
{
    fft2(psi, nx, ny, -1);
    double inv = 1.0 / ((double)nx * (double)ny);
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double ph = -0.5 * (kx[x] * kx[x] + ky[y] * ky[y]) * tau * 0.5;
            psi[(long)y * nx + x] *= (cos(ph) + I * sin(ph)) * inv;
        }
    fft2(psi, nx, ny, +1);
}

/* 2D form of the same scheme: K = (kx^2 + ky^2)/2, C = C_x (x) I + I (x) C_y,
 * e^{-iC tau} = e^{-iC_x tau} e^{-iC_y tau} (the two terms act on different
 * indices and commute), each by CN on every full-length row / column. */
int orc_step2d(int nx, int ny, long nsteps, cplx *psi, const double *kx, const double *ky,
               const cplx *U, const cplx *Cxs, const cplx *Cxd, const cplx *Cxu,
               const cplx *Cys, const cplx *Cyd, const cplx *Cyu, double tau)
{
    long np = (long)nx * ny;
    cplx *vh = (cplx *)malloc(sizeof(cplx) * np);
    if (!vh) return -2;
    for (long i = 0; i < np; ++i) vh[i] = cexp(-I * U[i] * tau * 0.5);
    int bad = 0;
    for (long s = 0; s < nsteps && !bad; ++s) {
        kinetic_half2(psi, nx, ny, kx, ky, tau);
        for (long i = 0; i < np; ++i) psi[i] *= vh[i];
        #pragma omp parallel reduction(|:bad)
        {
            int m = nx > ny ? nx : ny;
            cplx *work = (cplx *)malloc(sizeof(cplx) * 16 * m);
            cplx *col = (cplx *)malloc(sizeof(cplx) * m);
            #pragma omp for schedule(static)
            for (int y = 0; y < ny; ++y)
                if (cn_apply(nx, Cxs, Cxd, Cxu, tau, psi + (long)y * nx, work)) bad = 1;
            #pragma omp for schedule(static)
            for (int x = 0; x < nx; ++x) {
                for (int y = 0; y < ny; ++y) col[y] = psi[(long)y * nx + x];
                if (cn_apply(ny, Cys, Cyd, Cyu, tau, col, work)) bad = 1;
                for (int y = 0; y < ny; ++y) psi[(long)y * nx + x] = col[y];
            }
            free(work); free(col);
        }
        for (long i = 0; i < np; ++i) psi[i] *= vh[i];
        kinetic_half2(psi, nx, ny, kx, ky, tau);
    }
    free(vh);
    return bad ? -1 : 0;
}

/* --------------------------------------------------------------- 3D --- */
/* psi is [nz][ny][nx], x fastest.  A line of the grid along axis d starts
 * at `base` and has stride st[d]. */
static void line_get(const cplx *psi, long base, long stride, int n, cplx *line)
{
    for (int i = 0; i < n; ++i) line[i] = psi[base + (long)i * stride];
}

static void line_put(cplx *psi, long base, long stride, int n, const cplx *line)
{
    for (int i = 0; i < n; ++i) psi[base + (long)i * stride] = line[i];
}

/* the start of line j of the lines along axis d (j runs over the other two
 * indices, the faster one first) */
static long line_base(int d, long j, int nx, int ny)
{
    if (d == 0) return j * nx;                              /* j = z ny + y */
    if (d == 1) return (j / nx) * (long)nx * ny + j % nx;   /* j = z nx + x */
    return j;                                               /* j = y nx + x */
}

static void fft3(cplx *psi, const int *n, int sign)
{
    const long st[3] = {1, n[0], (long)n[0] * n[1]};
    const long np = (long)n[0] * n[1] * n[2];
    for (int d = 0; d < 3; ++d) {
        const long nl = np / n[d];
        #pragma omp parallel
        {
            cplx *line = (cplx *)malloc(sizeof(cplx) * n[d]);
            #pragma omp for schedule(static)
            for (long j = 0; j < nl; ++j) {
                const long b = line_base(d, j, n[0], n[1]);
                line_get(psi, b, st[d], n[d], line);
                orc_fft(line, n[d], sign);
                line_put(psi, b, st[d], n[d], line);
            }
            free(line);
        }
    }
}

static void kinetic_half3(cplx *psi, const int *n, const double *kx, const double *ky,
                          const double *kz, double tau)
{
    fft3(psi, n, -1);
    const double inv = 1.0 / ((double)n[0] * (double)n[1] * (double)n[2]);
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < n[2]; ++z)
        for (int y = 0; y < n[1]; ++y)
            for (int x = 0; x < n[0]; ++x) {
                double ph = -0.5 * (kx[x] * kx[x] + ky[y] * ky[y] + kz[z] * kz[z]) * tau * 0.5;
                psi[((long)z * n[1] + y) * n[0] + x] *= (cos(ph) + I * sin(ph)) * inv;
            }
    fft3(psi, n, +1);
}

/* 3D form of the scheme (the multidimensional case the paper names at the
 * end of Sec. V): K = (kx^2 + ky^2 + kz^2)/2, C = C_x + C_y + C_z as
 * Kronecker sums, e^{-iC tau} = e^{-iC_x tau} e^{-iC_y tau} e^{-iC_z tau}
 * (the three act on different indices and commute), each by CN on every
 * full-length line along its axis.  Cs, Cd, Cu hold the three axes' C
 * (sub, diag, super) one after another: x (nx each), then y, then z. */
int orc_step3d(int nx, int ny, int nz, long nsteps, cplx *psi, const double *kx,
               const double *ky, const double *kz, const cplx *U, const cplx *Cs,
               const cplx *Cd, const cplx *Cu, double tau)
{
    const int n[3] = {nx, ny, nz};
    const long st[3] = {1, nx, (long)nx * ny};
    const long np = (long)nx * ny * nz;
    const long coff[3] = {0, nx, (long)nx + ny};
    cplx *vh = (cplx *)malloc(sizeof(cplx) * np);
    if (!vh) return -2;
    for (long i = 0; i < np; ++i) vh[i] = cexp(-I * U[i] * tau * 0.5);
    int m = nx > ny ? nx : ny;
    if (nz > m) m = nz;
    int bad = 0;
    for (long s = 0; s < nsteps && !bad; ++s) {
        kinetic_half3(psi, n, kx, ky, kz, tau);
        for (long i = 0; i < np; ++i) psi[i] *= vh[i];
        for (int d = 0; d < 3; ++d) {
            const long nl = np / n[d];
            #pragma omp parallel reduction(|:bad)
            {
                cplx *work = (cplx *)malloc(sizeof(cplx) * 16 * m);
                cplx *line = (cplx *)malloc(sizeof(cplx) * m);
                #pragma omp for schedule(static)
                for (long j = 0; j < nl; ++j) {
                    const long b = line_base(d, j, nx, ny);
                    line_get(psi, b, st[d], n[d], line);
                    if (cn_apply(n[d], Cs + coff[d], Cd + coff[d], Cu + coff[d], tau, line, work))
                        bad = 1;
                    line_put(psi, b, st[d], n[d], line);
                }
                free(work); free(line);
            }
        }
        for (long i = 0; i < np; ++i) psi[i] *= vh[i];
        kinetic_half3(psi, n, kx, ky, kz, tau);
    }
    free(vh);
    return bad ? -1 : 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
