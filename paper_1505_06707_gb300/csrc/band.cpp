// Host construction of the ECS-friendly FFT preconditioner of Sec. III
// (Eqs. Prec_eigen_eq, K_l, PreconFFT_ECS): the band split, the band
// matrices K_l = 1/2 k_n k_m Q_{nm}, their eigen-decomposition (a small
// complex QR algorithm for the eigenvalues, inverse iteration for the
// eigenvectors) with the unconjugated normalisation chi^T chi = 1, and the
// per-axis tables the kernels read.
#include "band.h"

#include <algorithm>
#include <cmath>

namespace soft {

static const double PI_B = 3.14159265358979323846;

// Spectrum split of Sec. III (paragraph after Fig. 1), 0-based FFT order:
// {0}, bands of nbw on the positive side with the last (next to the Nyquist
// index) taking the remainder, {N/2}, the mirror image on the negative side.
std::vector<std::pair<int, int>> band_split(int n, int nbw) {
    std::vector<std::pair<int, int>> b;
    if (n < 4) {
        for (int m = 0; m < n; ++m) b.push_back({m, 1});
        return b;
    }
    const int half = n / 2, npos = half - 1;
    const int q = npos / nbw, r = npos % nbw;
    std::vector<int> w;
    if (q == 0) w.push_back(npos);
    else {
        for (int i = 0; i < q - 1; ++i) w.push_back(nbw);
        w.push_back(nbw + r);
    }
    b.push_back({0, 1});
    int m = 1;
    for (int x : w) { b.push_back({m, x}); m += x; }
    b.push_back({half, 1});
    for (auto it = w.rbegin(); it != w.rend(); ++it) { b.push_back({m + 1, *it}); m += *it; }
    return b;
}

// --- small dense complex linear algebra ------------------------------------
static void lu_solve(int n, std::vector<cd> A, std::vector<cd>& b) {
    std::vector<int> piv(n);
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (std::abs(A[i * n + k]) > std::abs(A[p * n + k])) p = i;
        if (p != k) {
            for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
            std::swap(b[k], b[p]);
        }
        cd d = A[k * n + k];
        if (d == 0.0) d = 1e-300;
        for (int i = k + 1; i < n; ++i) {
            const cd f = A[i * n + k] / d;
            if (f == 0.0) continue;
            for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        cd s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * b[j];
        cd d = A[i * n + i];
        if (d == 0.0) d = 1e-300;
        b[i] = s / d;
    }
}

// eigenvalues of a general complex matrix: Householder reduction to upper
// Hessenberg form, then single-shift QR with Wilkinson shifts and deflation
static int eigenvalues(int n, std::vector<cd> H, std::vector<cd>& lam) {
    // Hessenberg reduction
    for (int k = 0; k < n - 2; ++k) {
        double alpha = 0;
        for (int i = k + 1; i < n; ++i) alpha += std::norm(H[i * n + k]);
        alpha = std::sqrt(alpha);
        if (alpha == 0) continue;
        std::vector<cd> v(n, 0.0);
        const cd x0 = H[(k + 1) * n + k];
        const cd ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : cd(1.0);
        v[k + 1] = x0 + ph * alpha;
        for (int i = k + 2; i < n; ++i) v[i] = H[i * n + k];
        double vn = 0;
        for (int i = k + 1; i < n; ++i) vn += std::norm(v[i]);
        if (vn == 0) continue;
        // H <- (I - 2vv^H/vn) H (I - 2vv^H/vn)
        for (int j = 0; j < n; ++j) {
            cd s = 0;
            for (int i = k + 1; i < n; ++i) s += std::conj(v[i]) * H[i * n + j];
            s *= 2.0 / vn;
            for (int i = k + 1; i < n; ++i) H[i * n + j] -= v[i] * s;
        }
        for (int i = 0; i < n; ++i) {
            cd s = 0;
            for (int j = k + 1; j < n; ++j) s += H[i * n + j] * v[j];
            s *= 2.0 / vn;
            for (int j = k + 1; j < n; ++j) H[i * n + j] -= s * std::conj(v[j]);
        }
    }
    lam.assign(n, 0.0);
    int hi = n - 1, iter = 0;
    const double eps = 1e-15;
    while (hi >= 0) {
        if (hi == 0) { lam[0] = H[0]; --hi; continue; }
        int lo = hi;
        while (lo > 0) {
            const double s = std::abs(H[lo * n + lo]) + std::abs(H[(lo - 1) * n + lo - 1]);
            if (std::abs(H[lo * n + lo - 1]) <= eps * (s > 0 ? s : 1.0)) {
                H[lo * n + lo - 1] = 0.0;
                break;
            }
            --lo;
        }
        if (lo == hi) { lam[hi] = H[hi * n + hi]; --hi; iter = 0; continue; }
        if (++iter > 500) return -1;
        // Wilkinson shift from the trailing 2x2 block
        const cd a = H[(hi - 1) * n + hi - 1], b = H[(hi - 1) * n + hi];
        const cd c = H[hi * n + hi - 1], d = H[hi * n + hi];
        const cd tr = a + d, det = a * d - b * c;
        const cd disc = std::sqrt(tr * tr - 4.0 * det);
        cd m1 = 0.5 * (tr + disc), m2 = 0.5 * (tr - disc);
        cd mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
        if (iter % 11 == 10) mu += std::abs(H[hi * n + hi - 1]) * cd(0.75, 0.3);   // exceptional shift
        // QR step on the active window via Givens rotations
        std::vector<cd> cs(hi - lo), sn(hi - lo);
        for (int k = lo; k <= hi; ++k) H[k * n + k] -= mu;
        for (int k = lo; k < hi; ++k) {
            const cd x = H[k * n + k], y = H[(k + 1) * n + k];
            const double r = std::sqrt(std::norm(x) + std::norm(y));
            cd cc = 1.0, ss = 0.0;
            if (r > 0) { cc = x / r; ss = y / r; }
            cs[k - lo] = cc; sn[k - lo] = ss;
            for (int j = k; j < n; ++j) {        // rows k, k+1 <- G^H [row k; row k+1]
                const cd t1 = H[k * n + j], t2 = H[(k + 1) * n + j];
                H[k * n + j] = std::conj(cc) * t1 + std::conj(ss) * t2;
                H[(k + 1) * n + j] = -ss * t1 + cc * t2;
            }
        }
        for (int k = lo; k < hi; ++k) {          // columns k, k+1 <- [col k, col k+1] G
            const cd cc = cs[k - lo], ss = sn[k - lo];
            const int rmax = std::min(k + 2, hi);
            for (int i = 0; i <= rmax; ++i) {
                const cd t1 = H[i * n + k], t2 = H[i * n + k + 1];
                H[i * n + k] = t1 * cc + t2 * ss;
                H[i * n + k + 1] = -t1 * std::conj(ss) + t2 * std::conj(cc);
            }
        }
        for (int k = lo; k <= hi; ++k) H[k * n + k] += mu;
    }
    return 0;
}

// K v = lambda v: eigenvalues by QR, eigenvectors by two steps of inverse
// iteration, normalised by v^T v = 1 (unconjugated, Sec. III after Eq. K_l).
// Returns the largest residual |K v - lambda v| and |X^T X - I| entry.
int eig_complex_symmetric(int n, const std::vector<cd>& K, std::vector<cd>& lam,
                          std::vector<cd>& V /* n x n, column j = eigenvector j */,
                          double* resid, double* orth) {
    if (eigenvalues(n, K, lam)) return -1;
    V.assign((size_t)n * n, 0.0);
    double kn = 0;
    for (const cd& v : K) kn = std::max(kn, std::abs(v));
    if (kn == 0) kn = 1;
    for (int j = 0; j < n; ++j) {
        std::vector<cd> M = K;
        const cd shift = lam[j] + cd(1e-13 * kn, 1e-13 * kn);
        for (int i = 0; i < n; ++i) M[i * n + i] -= shift;
        std::vector<cd> v(n);
        for (int i = 0; i < n; ++i) v[i] = cd(1.0 + 0.1 * i, 0.37 * (i % 3) - 0.2);
        for (int it = 0; it < 3; ++it) {
            lu_solve(n, M, v);
            double s = 0;
            for (int i = 0; i < n; ++i) s += std::norm(v[i]);
            s = std::sqrt(s);
            for (int i = 0; i < n; ++i) v[i] /= s;
        }
        cd tt = 0;
        for (int i = 0; i < n; ++i) tt += v[i] * v[i];
        if (std::abs(tt) < 1e-8) return -2;      // quasi-null vector: chi^T chi ~ 0
        const cd sc = 1.0 / std::sqrt(tt);
        for (int i = 0; i < n; ++i) V[(size_t)i * n + j] = v[i] * sc;
    }
    double rmax = 0, omax = 0;
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) {
            cd s = 0;
            for (int k = 0; k < n; ++k) s += K[i * n + k] * V[(size_t)k * n + j];
            rmax = std::max(rmax, std::abs(s - lam[j] * V[(size_t)i * n + j]) / kn);
        }
        for (int l = 0; l < n; ++l) {
            cd s = 0;
            for (int k = 0; k < n; ++k) s += V[(size_t)k * n + j] * V[(size_t)k * n + l];
            omax = std::max(omax, std::abs(s - (j == l ? 1.0 : 0.0)));
        }
    }
    *resid = rmax;
    *orth = omax;
    return 0;
}

// Per-axis preconditioner tables.  simple = true gives Eq. PreconFFT
// (one-wide bands, X = identity, lambda = k^2/2); otherwise Eq.
// PreconFFT_ECS with N_BW = nbw.  The paper's F has F_nj = e^{i k_n x_j}/sqrt N;
// its phase e^{i k_n x_0}/sqrt N is folded into the rows of X (Xf) and
// e^{-i k_n x_0}/sqrt N into X^T (Xb).
int build_band_axis(const Axis1D& A, int nbw, bool simple, BandAxis& out, double* check) {
    const int n = A.n;
    const double L = A.b - A.a;
    out.n = n;
    out.lam.assign(n, 0.0);
    out.start.assign(n, 0);
    out.width.assign(n, 1);
    out.xf.clear(); out.xb.clear(); out.off.assign(n, 0);
    *check = 0;
    auto bands = simple ? std::vector<std::pair<int, int>>() : band_split(n, nbw);
    if (simple)
        for (int m = 0; m < n; ++m) bands.push_back({m, 1});
    int wmax = 1;
    for (auto& b : bands) wmax = std::max(wmax, b.second);
    // g(d) = (1/N) sum_j e^{2 pi i d x_j/L} q_j^-2 (grid quadrature of Q)
    std::vector<cd> g(2 * wmax + 1, 0.0);
    for (int d = -wmax; d <= wmax; ++d) {
        cd s = 0;
        for (int j = 0; j < n; ++j) s += std::polar(1.0, 2 * PI_B * d * A.x[j] / L) / (A.q[j] * A.q[j]);
        g[d + wmax] = s / (double)n;
    }
    const double x0 = A.x[0], rn = 1.0 / std::sqrt((double)n);
    for (auto& b : bands) {
        const int m0 = b.first, w = b.second;
        std::vector<cd> K((size_t)w * w), lam, V;
        if (simple) {
            lam.assign(1, 0.5 * A.k[m0] * A.k[m0]);
            V.assign(1, 1.0);
        } else {
            for (int u = 0; u < w; ++u)
                for (int v = 0; v < w; ++v)
                    K[(size_t)u * w + v] = 0.5 * A.k[m0 + u] * A.k[m0 + v] * g[(v - u) + wmax];
            double res, orth;
            if (eig_complex_symmetric(w, K, lam, V, &res, &orth)) return SOFT_ERR_SETUP;
            if (res > 1e-10 || orth > 1e-9) return SOFT_ERR_SETUP;
            *check = std::max(*check, std::max(res, orth));
        }
        // rows of X are the eigenvectors: X[nu][m] = V[m][nu]
        for (int u = 0; u < w; ++u) {
            const int nu = m0 + u;
            out.lam[nu] = lam[u];
            out.start[nu] = m0;
            out.width[nu] = w;
            out.off[nu] = (int)out.xf.size();
            for (int v = 0; v < w; ++v) {
                const int m = m0 + v;
                // forward: c_nu = sum_m X[nu][m] e^{i k_m x0}/sqrt N (sum_j e^{2 pi i m j/N} r_j)
                out.xf.push_back(V[(size_t)v * w + u] * std::polar(rn, A.k[m] * x0));
                // backward: d_m = e^{-i k_m x0}/sqrt N sum_nu X[nu][m] c_nu, stored per output m
                out.xb.push_back(V[(size_t)u * w + v] * std::polar(rn, -A.k[nu] * x0));
            }
        }
    }
    return SOFT_OK;
}

}  // namespace soft
