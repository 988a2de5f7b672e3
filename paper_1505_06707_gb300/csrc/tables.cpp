// Host FP64 construction of the per-problem tables of the GPU library:
// grid, momenta, contour, potential, the absorbing matrix C and the
// factorisation used by the strip Crank-Nicolson solve.  Everything follows
// Serov & Sergeeva, arXiv:1505.06707, Sec. II (grid Eq. DVRgrid, momenta
// after Eq. FFTbasis, contour Eq. ECSintdef, K_s Eq. Ks_FD, K_FD Eq. K_FD,
// C Eq. C_FD) and Sec. IV (the contours).
#include "host_tables.h"

#include <cmath>

namespace soft {

static const double PI = 3.14159265358979323846;

ContourFn::ContourFn(int kind, double R0, double rmax, double theta, double alpha, double e_cap,
                     double kmin)
    : kind(kind), R0(R0), rmax(rmax), theta(theta), alpha(alpha), e_cap(e_cap), kmin(kmin) {}

// comparison absorbers of Sec. IV (the contour stays real): the linear CAP
// U_a = E_CAP [1 - q^2] with the SECS q (Eq. CAP_via_q) and TFAP
// U_a = -i (k_min^2/2) y(s) (Eqs. TFAP, yTFAP), zero for |x| <= R0
cd ContourFn::absorber(double x) const {
    const double ax = std::fabs(x);
    if (ax <= R0) return 0.0;
    const double s = (ax - R0) / (rmax - R0);
    if (kind == SOFT_ABSORB_CAP) {
        const cd qq = std::polar(1.0, theta * s);
        return e_cap * (1.0 - qq * qq);
    }
    if (kind == SOFT_ABSORB_TFAP) {
        const double c = 2.622057, a = c * c * c - 16.0, b = c * c * c - 17.0;
        const double y = (a * s - b * s * s * s + 4.0 / ((1 - s) * (1 - s)) - 4.0 / ((1 + s) * (1 + s))) / (c * c);
        return cd(0.0, -0.5 * kmin * kmin * y);
    }
    return 0.0;
}

// q(x); returns false where q is infinite (TFECS at |x| = rmax)
bool ContourFn::q(double x, cd* out) const {
    const double ax = std::fabs(x);
    if (ax <= R0 || kind == SOFT_ABSORB_CAP || kind == SOFT_ABSORB_TFAP) { *out = 1.0; return true; }
    const double s = (ax - R0) / (rmax - R0);
    switch (kind) {
    case SOFT_CONTOUR_SHARP: *out = std::polar(1.0, theta); return true;
    case SOFT_CONTOUR_SECS: *out = std::polar(1.0, theta * s); return true;
    case SOFT_CONTOUR_TFECS: {
        if (s >= 1.0) return false;
        const double y = alpha * (1.0 / ((1 - s) * (1 - s)) - 1.0 / ((1 + s) * (1 + s)) - 4 * s);
        *out = std::sqrt(cd(1.0, y));
        return true;
    }
    }
    *out = 1.0;
    return true;
}

cd ContourFn::inv_q(double x) const {
    cd v;
    return q(x, &v) ? 1.0 / v : cd(0.0);
}

// 16-point Gauss-Legendre nodes and weights on [-1, 1]
static const double GL_X[8] = {0.0950125098376374, 0.2816035507792589, 0.4580167776572274,
                               0.6178762444026438, 0.7554044083550030, 0.8656312023878318,
                               0.9445750230732326, 0.9894009349916499};
static const double GL_W[8] = {0.1894506104550685, 0.1826034150449236, 0.1691565193950025,
                               0.1495959888165767, 0.1246289712555339, 0.0951585116824928,
                               0.0622535239386479, 0.0271524594117541};

// z(x) = int_0^x q (Eq. ECSintdef)
cd ContourFn::z(double x) const {
    const double ax = std::fabs(x), sg = x < 0 ? -1.0 : 1.0;
    if (ax <= R0 || kind == SOFT_ABSORB_CAP || kind == SOFT_ABSORB_TFAP) return x;
    const double d = ax - R0;
    switch (kind) {
    case SOFT_CONTOUR_SHARP: return sg * (R0 + std::polar(1.0, theta) * d);
    case SOFT_CONTOUR_SECS: {
        // (W/(i theta)) (e^{i phi} - 1) with phi = theta d/W, written as
        // d sinc(phi/2) e^{i phi/2}: no cancellation for small theta, and
        // theta = 0 gives the unscaled z = x
        const double ph = theta * d / (rmax - R0);
        const double sinc = ph == 0.0 ? 1.0 : std::sin(0.5 * ph) / (0.5 * ph);
        return sg * (R0 + d * sinc * std::polar(1.0, 0.5 * ph));
    }
    case SOFT_CONTOUR_TFECS: {
        // q grows like 1/(1-s) towards s = 1; with s = 1 - e^{-u} the
        // integrand q(s) e^{-u} du is smooth, so composite Gauss-Legendre on
        // pieces of length <= 1/4 in u converges to round-off
        const double W = rmax - R0;
        const double umax = -std::log1p(-d / W);
        const int pieces = 1 + (int)std::ceil(4.0 * umax);
        const double du = umax / pieces;
        cd acc = 0.0;
        for (int p = 0; p < pieces; ++p) {
            const double c = (p + 0.5) * du, hw = 0.5 * du;
            for (int k = 0; k < 8; ++k)
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    const double u = c + sgn * hw * GL_X[k];
                    const double e = std::exp(-u);
                    cd qq;
                    q(R0 + W * (1.0 - e), &qq);
                    acc += GL_W[k] * hw * qq * e;
                }
        }
        return sg * (R0 + W * acc);
    }
    }
    return x;
}

void build_axis(Axis1D& A, int n, double a, double b, const ContourFn& cf, double tau) {
    A.n = n; A.a = a; A.b = b;
    A.h = (b - a) / n;
    A.x.resize(n); A.k.resize(n); A.q.resize(n); A.z.resize(n);
    const double L = b - a;
    for (int j = 0; j < n; ++j) {
        A.x[j] = a + A.h * (j + 0.5);
        A.k[j] = (j < n / 2) ? 2 * PI * j / L : -2 * PI * (n - j) / L;
        cd qq;
        if (!cf.q(A.x[j], &qq)) qq = 1e300;   // not reached: grid points avoid |x| = rmax
        A.q[j] = qq;
        A.z[j] = cf.z(A.x[j]);
    }
    // C = K_s - K_FD (Eq. C_FD), periodic; Eq. Ks_FD with midpoints x_{j+1/2} = a + h(j+1)
    std::vector<cd> qh(n), iqm(n);
    for (int j = 0; j < n; ++j) {
        qh[j] = 1.0 / std::sqrt(A.q[j]);                  // q_j^{-1/2}, principal branch
        iqm[j] = cf.inv_q(a + A.h * (j + 1));             // 1/q_{j+1/2}
    }
    const double c = -0.5 / (A.h * A.h);
    A.Cs.resize(n); A.Cd.resize(n); A.Cu.resize(n);
    // the coupling of j and j+1 is one product, stored as C[j][j+1] and
    // C[j+1][j], so that C is symmetric to the last bit (the strip solve
    // uses one multiplier array for both sweeps)
    for (int j = 0; j < n; ++j) {
        const int jm = (j + n - 1) % n, jp = (j + 1) % n;
        const cd e = c * qh[j] * qh[jp] * iqm[j] - c;
        const cd dia = -c * qh[j] * qh[j] * (iqm[j] + iqm[jm]);
        A.Cu[j] = e;
        A.Cs[jp] = e;
        A.Cd[j] = dia + 2.0 * c;
    }
    A.tau = tau;
}

// Strip block: complement of the longest cyclic run of rows where C vanishes.
int find_block(const Axis1D& A, int* blk0, int* nb) {
    const int n = A.n;
    std::vector<char> nz(n);
    int cnt = 0;
    for (int j = 0; j < n; ++j) {
        nz[j] = (A.Cs[j] != 0.0 || A.Cd[j] != 0.0 || A.Cu[j] != 0.0);
        cnt += nz[j];
    }
    if (cnt == 0) { *blk0 = 0; *nb = 0; return SOFT_OK; }
    if (cnt == n) return SOFT_ERR_SETUP;      // no unscaled interior
    // longest cyclic run of zero rows
    int best = 0, bstart = 0;
    for (int s = 0; s < n; ++s) {
        if (nz[s] || !nz[(s + n - 1) % n]) continue;   // run starts after a non-zero row
        int len = 0;
        while (len < n && !nz[(s + len) % n]) ++len;
        if (len > best) { best = len; bstart = s; }
    }
    *blk0 = (bstart + best) % n;
    *nb = n - best;
    return SOFT_OK;
}

// Tridiagonal solve with partial pivoting (reference for the self-check).
static void tri_pivot_solve(std::vector<cd> dl, std::vector<cd> d, std::vector<cd> du,
                            std::vector<cd>& b) {
    const int n = (int)d.size();
    std::vector<cd> du2(n, 0.0);
    for (int i = 0; i < n - 1; ++i) {
        if (std::abs(d[i]) >= std::abs(dl[i])) {
            const cd f = dl[i] / d[i];
            d[i + 1] -= f * du[i];
            b[i + 1] -= f * b[i];
        } else {
            const cd f = d[i] / dl[i];
            const cd di1 = d[i + 1];
            const cd dui1 = (i < n - 2) ? du[i + 1] : cd(0.0);
            d[i] = dl[i];
            const cd odu = du[i];
            du[i] = di1;
            du2[i] = dui1;
            d[i + 1] = odu - f * di1;
            if (i < n - 2) du[i + 1] = -f * dui1;
            const cd bi = b[i];
            b[i] = b[i + 1];
            b[i + 1] = bi - f * b[i + 1];
        }
    }
    b[n - 1] /= d[n - 1];
    if (n > 1) b[n - 2] = (b[n - 2] - du[n - 2] * b[n - 1]) / d[n - 2];
    for (int i = n - 3; i >= 0; --i) b[i] = (b[i] - du[i] * b[i + 1] - du2[i] * b[i + 2]) / d[i];
}

// LU (no pivoting) of M = 1 + i tau C/2 on the block, as the recurrences the
// kernels run: y_i = mf_i y_{i-1} + r_i ; x_i = mb_i x_{i+1} + g_i y_i.
int strip_factor(const Axis1D& A, int blk0, int nb, std::vector<cd>& mf, std::vector<cd>& mb,
                 std::vector<cd>& g, double* check_err) {
    const int n = A.n;
    const cd ih(0.0, 0.5 * A.tau);
    std::vector<cd> dl(std::max(nb - 1, 0)), d(nb), du(std::max(nb - 1, 0));
    for (int i = 0; i < nb; ++i) {
        const int j = (blk0 + i) % n;
        d[i] = 1.0 + ih * A.Cd[j];
        if (i + 1 < nb) {
            du[i] = ih * A.Cu[j];
            dl[i] = ih * A.Cs[(j + 1) % n];
        }
    }
    mf.assign(nb, 0.0); mb.assign(nb, 0.0); g.assign(nb, 0.0);
    std::vector<cd> delta(nb);
    delta[0] = d[0];
    for (int i = 1; i < nb; ++i) {
        const cd l = dl[i - 1] / delta[i - 1];
        mf[i] = -l;
        delta[i] = d[i] - l * du[i - 1];
    }
    for (int i = 0; i < nb; ++i) {
        if (delta[i] == 0.0) return SOFT_ERR_SETUP;
        g[i] = 1.0 / delta[i];
        if (i + 1 < nb) mb[i] = -du[i] / delta[i];
    }
    // self-check against a pivoted solve on a deterministic right-hand side
    std::vector<cd> r(nb), y(nb), x(nb);
    for (int i = 0; i < nb; ++i) r[i] = cd(std::cos(0.37 * i + 0.1), std::sin(1.13 * i));
    y[0] = r[0];
    for (int i = 1; i < nb; ++i) y[i] = mf[i] * y[i - 1] + r[i];
    x[nb - 1] = g[nb - 1] * y[nb - 1];
    for (int i = nb - 2; i >= 0; --i) x[i] = mb[i] * x[i + 1] + g[i] * y[i];
    std::vector<cd> ref = r;
    tri_pivot_solve(dl, d, du, ref);
    double num = 0, den = 0;
    for (int i = 0; i < nb; ++i) { num += std::norm(x[i] - ref[i]); den += std::norm(ref[i]); }
    *check_err = std::sqrt(num / std::max(den, 1e-300));
    return *check_err < 1e-12 ? SOFT_OK : SOFT_ERR_SETUP;
}

static std::vector<int> pass_radices(int logn, int logrm) {
    std::vector<int> lr;
    for (int p = 0; p < logn / logrm; ++p) lr.push_back(logrm);
    if (logn % logrm) lr.push_back(logn % logrm);
    return lr;
}

// Twiddle bases of the in-place FFT passes: for pass p (length L, stride
// s = L/R) four rows of s values, row k holding W_L^{off 2^k} for off < s.
std::vector<cd> pass_twiddles(int logn, int logrm) {
    std::vector<cd> out;
    int logl = logn;
    for (int lr : pass_radices(logn, logrm)) {
        const int L = 1 << logl, s = 1 << (logl - lr);
        for (int k = 0; k < 4; ++k)          // row k: W_L^{2^k off}, off < s
            for (int off = 0; off < s; ++off) {
                const long e = (long)off << k;
                const double ang = -2.0 * PI * (double)(e % L) / (double)L;
                out.push_back(cd(std::cos(ang), std::sin(ang)));
            }
        logl -= lr;
    }
    return out;
}

// The same passes with every twiddle W_L^{M off} (rows M = 1 .. R-1, off < s)
// for passes whose stride s satisfies 1 < s <= full_maxs, and four rows
// W_L^{M off}, M = 1 .. 4, otherwise (the complex128 1D step's layout).
std::vector<cd> pass_twiddles_full(int logn, int logrm, int full_maxs) {
    std::vector<cd> out;
    int logl = logn;
    for (int lr : pass_radices(logn, logrm)) {
        const int L = 1 << logl, s = 1 << (logl - lr), R = 1 << lr;
        const bool full = s > 1 && s <= full_maxs;
        const int rows = full ? R - 1 : 4;
        for (int r = 0; r < rows; ++r)
            for (int off = 0; off < s; ++off) {
                const long e = (long)(r + 1) * off;
                const double ang = -2.0 * PI * (double)(e % L) / (double)L;
                out.push_back(cd(std::cos(ang), std::sin(ang)));
            }
        logl -= lr;
    }
    return out;
}

// mixed-radix digit reversal of the in-place DIF FFT with passes of radix
// 2^logrm and a final radix 2^(logn mod logrm): position n holds frequency perm[n]
std::vector<int> dif_output_order(int logn, int logrm) {
    const std::vector<int> lr = pass_radices(logn, logrm);
    const int N = 1 << logn;
    std::vector<int> perm(N);
    for (int n = 0; n < N; ++n) {
        int rem = n, L = N, mult = 1, k = 0;
        for (int l : lr) {
            const int R = 1 << l, s = L / R;
            const int m = rem / s;
            rem %= s;
            k += m * mult;
            mult *= R;
            L = s;
        }
        perm[n] = k;
    }
    return perm;
}

cd soft_coulomb(const cd* z, int nd, double a2, double Z) {
    cd s = a2;
    for (int d = 0; d < nd; ++d) s += z[d] * z[d];
    return -Z / std::sqrt(s);
}

}  // namespace soft
